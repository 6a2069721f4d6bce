"""GB300-native matrix-free Hubbard exact diagonalisation in the one-spin-configuration basis.

The CUDA library is loaded lazily by :mod:`paper_1307_7542_gb300.hub`; importing the
package itself loads nothing.
"""
__all__ = ["hub", "workloads"]
