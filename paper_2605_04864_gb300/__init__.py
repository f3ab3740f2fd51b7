"""GB300-native FFT multipole estimators (Yamamoto P_l with m >= 0 symmetry, modified P_lb,
Scoccimarro B_l and the compressed TripoSH B_l0l with analytic shot noise).

The compute path is libnpc.so (hand-written CUDA for sm_103a, C ABI in include/npc.h);
``binding`` exposes that ABI with the same names and ``api`` is a thin NumPy/torch front end.
"""
__all__ = ["binding", "api", "autograd"]
