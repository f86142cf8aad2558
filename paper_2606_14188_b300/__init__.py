"""B300-native contact-smoothed differentiable rope/cloth simulator (arxiv 2606.14188, Sec. 4.1).

The compute path is the C-ABI library libcordsim.so (hand-written CUDA for sm_103a); the Python
modules here only marshal arguments.  `scenes` is the seeded input generator.
"""
