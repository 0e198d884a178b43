"""GB300 (sm_103a) recursive camera painting (arXiv 2312.12392).

    from paper_2312_12392_gb300 import rcp      # C-ABI binding (librcp.so)
    from paper_2312_12392_gb300 import scenes   # seeded synthetic workloads

The compute path is the CUDA library built by ``paper_2312_12392_gb300.build``;
importing the package does not load it (``rcp.lib()`` does, and fails loudly if
it was not built).
"""
__all__ = ["rcp", "scenes", "build"]
