"""GB300-native explicit upwind-DG convection step (arXiv:1508.04245).

``dgconv`` is the binding of the CUDA library (loaded on first use);
``workloads`` holds the seeded synthetic inputs.
"""
