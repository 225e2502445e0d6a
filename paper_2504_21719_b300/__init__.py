"""B300-native (sm_103a) SBR radio maps: Fibonacci-lattice ray launch, BVH
construction (Karras LBVH or binned SAH) and traversal, Fresnel / slab
interactions and plane deposit in hand-written CUDA kernels behind the C ABI
of include/rmsbr.h.

``paper_2504_21719_b300.api`` holds the PyTorch-facing helpers; importing it
loads librmsbr.so and fails loudly if the library has not been built.
"""
__all__ = ["api", "build"]
