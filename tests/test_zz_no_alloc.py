"""vie_matvec_noalloc: the Tucker matvec for callers that cannot allocate
device memory when they need a product (serving loops whose memory belongs to
another allocator under a fixed budget, callbacks that must not trigger the
synchronisation of cudaMalloc/cudaFree).

It must give what vie_matvec gives (same tolerance as the other FP32 matvec
tests, 1e-5 relative L2) on consecutive calls that share its fixed scratch
array, agree with the FP64 oracle's FFT matvec, change no device memory use
after its first call, and refuse sizes beyond that array with VIE_ERR_ARG.
This file is collected last on purpose.
"""
import ctypes

import numpy as np

from oracle import embed, kernel, matvec
import pytest
import torch

vie = pytest.importorskip("paper_1811_00484_gb300")
pytestmark = pytest.mark.gpu


def _field(n, B, seed):
    rng = np.random.default_rng(seed)
    shape = (B, 3) + tuple(n)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return torch.from_numpy(a.astype(np.complex64)).cuda()


def _noalloc(op, J, Y, B):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return vie.lib.vie_matvec_noalloc(op._h, ctypes.c_void_p(J.data_ptr()),
                                      ctypes.c_void_p(Y.data_ptr()), B, stream)


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("n,B", [((16, 16, 16), 2), ((12, 10, 20), 1)])
def test_noalloc_matches_matvec_on_consecutive_calls(n, B):
    op = vie.Operator(n, 5e-3, 298e6, 1e-6)
    for call, seed in enumerate((11, 12)):
        J = _field(n, B, seed)
        ref = op.matvec(J)
        Y = torch.empty_like(J)
        if call == 1:
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
        assert _noalloc(op, J, Y, B) == 0, vie.lib.vie_last_error().decode()
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert _rel(Y, ref) <= 1e-5
        if call == 1:
            # against the oracle's FFT matvec on the uncompressed spectra: FP32
            # rounding plus the HOSVD truncation (tol 1e-6, eq. (12))
            G = embed.green_spectra(kernel.toeplitz_tensor(*n, 5e-3, kernel.wavenumber(298e6)), *n)
            Jh = J.cpu().numpy().astype(np.complex128)
            yo = matvec.matvec_fft(G, Jh)
            yg = Y.cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) <= 1e-5 + 4e-6
    op.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = (64, 64, 64)                       # 37.7 MB per right-hand side
    op = vie.Operator(n, 5e-3, 298e6, 1e-6)
    J = _field(n, 2, 3)
    Y = torch.empty_like(J)
    assert _noalloc(op, J, Y, 2) == 1
    assert "scratch" in vie.lib.vie_last_error().decode()
    assert _noalloc(op, J[:1].contiguous(), Y[:1].contiguous(), 1) == 0
    op.close()
