"""FP64 CPU oracle for the Tucker-compressed FFT-VIE operator and its solve.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import or run anything here.  The CUDA library never calls it, and it never
calls the CUDA library: the two share no code.  Inputs come from the
separate ``workloads`` module, which holds no arithmetic of the method.

Everything is plain NumPy/SciPy in complex128, written to be read against
the paper (Giannakopoulos, Litsarev, Polimeridis, "Memory footprint
reduction for the FFT-based volume integral equation method via tensor
decompositions"):

  kernel.py   eqs. (5)-(6): the dyadic kernel (k0^2 I + grad grad) g sampled on
              the voxel grid, with an equivalent-sphere self term.
  embed.py    Section II.B and V.A: circulant embedding of the Toeplitz
              defining tensor and its 3-D DFT.
  matvec.py   Section II.B / V.B: the BTTB matrix-vector product, brute force
              and via FFT; the J-block system operator of eq. (4).
  hosvd.py    Algorithm 1 (HOSVD), eqs. (13)-(14), Definitions A.2-A.3.
  cp.py       Algorithm 2 (Tucker+CP: CP-ALS on the HOSVD core), eq. (17).
  factorwise.py  Section V.A: embedding and DFT applied to the Tucker factors.
  gmres.py    Section VI.C: restarted GMRES.
  adjoint.py  adjoint operator and the contrast gradient of a field misfit.

Readings of the paper where it is silent or garbled are listed in each
function's docstring.  Parity is pinned by ``tests/test_oracle_*.py``; the
equivalent-sphere self term and the point-sampled off-diagonal entries are a
stand-in for the paper's Galerkin PWL integrals, whose physics fidelity is
parity unpinned (only the formulas themselves are pinned).
"""
from . import kernel, embed, matvec, hosvd, cp, factorwise, gmres, adjoint  # noqa: F401
