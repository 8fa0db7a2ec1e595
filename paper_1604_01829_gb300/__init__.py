"""GB300-native lattice Boltzmann + raspberry-colloid coupling (sm_103a).

The hot path (fused D3Q19 collide-and-stream, bead coupling, rigid bodies)
runs in the CUDA library behind the C ABI of include/lb.h; ``lb`` is its
Python binding and ``workloads`` generates seeded inputs shaped like the
paper's (Ustach & Faller, arXiv:1604.01829).
"""
