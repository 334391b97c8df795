"""FP64 CPU oracle for the BLWS path (Lin & Wei, "A Block Lanczos with Warm Start
Technique for Accelerating Nuclear Norm Minimization Algorithms").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything in this package.  The product path (the CUDA library
under ``paper_1012_0365_gb300``) never calls it, and this package never imports
the product.  The two share no code: only the seeded input generators in
``paper_1012_0365_gb300.synthetic`` feed both, and those hold none of the
method's arithmetic.

Everything here is plain, slow and FP64: NumPy (LAPACK through OpenBLAS) for
library primitives, plus a plain-C one-sided Jacobi SVD (``jacobi_svd.c``) used
only as an independent brute-force check on tiny inputs.

Modules
-------
svt      Eq. (3)-(4): the shrinkage operator and SVT by full SVD.
lanczos  Algorithm 1: the single-vector Lanczos procedure (b = 1 pin).
blws     Eq. (7)-(13), Algorithms 2 and 3, Theorem 1, Section 4: block
         Lanczos on the augmented matrix with the mixed warm start, and
         BL_EVD of a symmetric matrix with a warm start.
rpca     Section 5 host: inexact ALM Robust PCA with full-SVD SVT.
mc       Section 5 host: SVT matrix completion, and the proximal (FPC-type)
         variant whose W is a sparse residual plus a low-rank term.
cjacobi  ctypes loader for the C Jacobi SVD.
"""

from .svt import theta, svt_full, svt_factored  # noqa: F401
from .lanczos import lanczos_alg1  # noqa: F401
from .blws import (augmented, apply_augmented, block_lanczos, assemble_T,  # noqa: F401
                   bl_evd, blws_svt_ref, cold_svt_ref, warm_start_block,
                   qr_deflate, blws_evd_ref)
from .rpca import rpca_ialm_full, rpca_ialm_blws, rank_predict  # noqa: F401
from .mc import mc_svt_full, mc_prox_full  # noqa: F401
