"""The rank-versus-frequency sweep of Sec. VI.A (Fig. 4; `bench.py --mode ranks`)
at its three lowest frequencies, resolution lambda/10, on a cube of unit edge:
the device HOSVD ranks at tol 1e-8 equal the oracle's (Algorithm 1 on the
FP64 spectra; a rank may differ only where a discarded tail lies within
1e-9 of the threshold), and the maximum rank grows with frequency."""
import math

import numpy as np
import pytest

from oracle import embed as E
from oracle import hosvd as H
from oracle import kernel as K

vie = pytest.importorskip("paper_1811_00484_gb300")
pytestmark = pytest.mark.gpu

C0 = 299792458.0


def test_max_rank_grows_with_frequency_and_matches_the_oracle():
    tol = 1e-8
    maxima = []
    for i in (1, 2, 3):
        f = 0.3e9 * i
        n = round(10 / (C0 / f))
        h = 1.0 / n
        op = vie.Operator((n, n, n), h, f, tol)
        ranks = op.info()["ranks"]
        op.close()
        Ghat = E.green_spectra(K.toeplitz_tensor(n, n, n, h, K.wavenumber(f)), n, n, n)
        for c in range(6):
            A = Ghat[c]
            norm_A = H.frobenius(A)
            for q in range(3):
                s = np.linalg.svd(H.unfold(A, q), compute_uv=False)
                r = H.truncation_rank(s, tol, norm_A, "tail")
                if ranks[c][q] != r:
                    k = min(r, ranks[c][q])
                    tail = math.sqrt(float(np.sum(s[k:] ** 2)))
                    assert abs(tail - tol / math.sqrt(3) * norm_A) <= 1e-9 * s[0], (f, c, q)
        maxima.append(max(max(r) for r in ranks))
    assert maxima[0] < maxima[1] < maxima[2]
