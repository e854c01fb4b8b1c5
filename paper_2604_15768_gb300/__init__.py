"""GB300-native coupled-configuration generation, de-duplication and
variational energy for selected-CI with neural-network quantum states.

The compute path is the CUDA library ``libcusci`` behind the C-ABI declared in
``include/cusci.h``; ``paper_2604_15768_gb300.cusci`` binds it.
"""
