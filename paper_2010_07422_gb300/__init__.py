"""IRCUR (Iterated Robust CUR, arXiv 2010.07422) on GB300: a C-ABI CUDA
library (libircur.so, built from csrc/) and its Python binding (ircur.py).

    from paper_2010_07422_gb300 import ircur
    solver = ircur.IRCUR(n1, n2, r, resample=True)
"""

__all__ = ["ircur", "synth", "build"]
