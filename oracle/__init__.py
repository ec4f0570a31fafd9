"""Plain FP64 CPU oracle for the accelerated divide-and-conquer (ADC) tridiagonal
eigensolver of Li, Liao, Liu and Jiang.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product path (``paper_1510_04591_gb300``) never imports it, and this package
never imports the product path: the two share no code.  The only module both
sides use is the seeded input generator ``paper_1510_04591_gb300.inputs``,
which holds none of the method's arithmetic (and is not imported here either:
callers pass arrays in).

Contents
--------
``dc``    : Cuppen/Gu-Eisenstat divide and conquer (Sec. 2.3, Algorithm 1) with
            the plain dense eigenvector update, built on the C routines in
            ``tdeig_oracle.c`` (leaf QR, deflation, secular roots, Loewner
            recomputation, Cauchy-like eigenvector matrix).
``hss``   : off-diagonal rank estimate (eq. bounds, Sec. 4.1), randomized HSS
            construction (Algorithm 2), SRRSC-style construction (ADC1) and
            HSS-times-matrix from the right (Algorithm 3), plus densification.
``metrics``: orthogonality and backward-error measures of Sec. 5, Example 3.

Parity status per function is listed in each module's docstring.
"""
from .clib import lib, build_oracle  # noqa: F401
