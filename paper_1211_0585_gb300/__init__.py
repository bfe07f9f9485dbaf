"""GB300-native messenger-field Wiener filter for HEALPix CMB maps
(Elsner & Wandelt, arXiv:1211.0585).

The compute path lives in a C-ABI shared library built from csrc/ (CUDA for
sm_103a); `paper_1211_0585_gb300.wf` is its thin ctypes binding. Importing the
package loads nothing; the library is opened on first use and its absence is
an error, never a fallback.
"""
__all__ = ["wf", "inputs"]
