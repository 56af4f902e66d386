"""GB300-native simplified DUGKS (S-DUGKS, arXiv:2007.07347) D2Q9 step.

``meshes`` holds the seeded input generators; ``sdugks`` the ctypes binding of the
CUDA library (imported lazily so that the generators load without a GPU).
"""
__all__ = ["meshes"]
