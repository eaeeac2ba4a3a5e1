"""B300-native analytic linac source model in use (arXiv:1503.01725).

The compute path is liblsm.so (CUDA, sm_103a), reached through the C ABI in
include/lsm.h; ``paper_1503_01725_b300.lsm`` is its Python binding and
``paper_1503_01725_b300.workloads`` draws seeded synthetic inputs.
"""
