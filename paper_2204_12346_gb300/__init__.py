"""GB300-native SIRD calibration by particle swarm optimisation (arXiv 2204.12346).

The compute path lives in a CUDA library behind a C ABI (``include/sird_pso.h``);
``paper_2204_12346_gb300.sird`` is its Python binding.  The binding is imported
lazily so that the synthetic-input helpers load without a GPU.
"""
