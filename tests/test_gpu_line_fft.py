"""The FP32 line-FFT engine on every supported length, through its C-ABI test
entry (one forward or inverse DFT per line, unnormalised).

Plans: one stage for N <= 16, two Stockham stages for 32..256, three for 512
and 1024 (16 elements per thread throughout).  The bar is the FP32 engine's:
rel-L2 per line <= 1e-6 against numpy's FP64 FFT (each value passes through
~log2(N) rounded butterflies and at most two rounded twiddle products, so the
error is a few times 1e-7).
"""
import numpy as np
import pytest

from paper_1909_08354_b300 import sn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = [8, 16, 32, 64, 128, 256, 512, 1024]


def lines(n, nlines, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nlines, n)) + 1j * rng.standard_normal((nlines, n))
    x *= np.exp(rng.uniform(-3, 3, (nlines, 1)))
    x[0] = 0
    x[1] = 0
    x[1, n // 3] = 1.5 + 0.5j  # a delta: a pure twiddle pattern out
    x[2] = 0.25 - 0.75j        # a constant: one nonzero bin out
    return x.astype(np.complex64)


@pytest.mark.parametrize("sign", [-1, 1])
@pytest.mark.parametrize("n", SIZES)
def test_line_dft_matches_numpy(n, sign):
    x = lines(n, 37, seed=n + sign)
    d = torch.from_numpy(x.copy()).cuda()
    sn.sn_test_line_fft_f32(d, n, sign, sn.SN_ENGINE_FP32)
    got = d.cpu().numpy().astype(np.complex128)
    xd = x.astype(np.complex128)
    ref = np.fft.fft(xd, axis=1) if sign < 0 else np.fft.ifft(xd, axis=1) * n
    for i in range(x.shape[0]):
        nrm = np.linalg.norm(ref[i])
        err = np.linalg.norm(got[i] - ref[i])
        assert err <= 1e-6 * nrm or (nrm == 0 and err == 0), (n, sign, i, err / max(nrm, 1e-300))


@pytest.mark.parametrize("n", [512, 1024])
def test_forward_then_inverse_is_n_times_identity(n):
    x = lines(n, 21, seed=5 * n)
    d = torch.from_numpy(x.copy()).cuda()
    sn.sn_test_line_fft_f32(d, n, -1, sn.SN_ENGINE_FP32)
    sn.sn_test_line_fft_f32(d, n, 1, sn.SN_ENGINE_FP32)
    got = d.cpu().numpy().astype(np.complex128) / n
    xd = x.astype(np.complex128)
    for i in range(x.shape[0]):
        nrm = np.linalg.norm(xd[i])
        err = np.linalg.norm(got[i] - xd[i])
        assert err <= 2e-6 * nrm or (nrm == 0 and err == 0), (n, i, err / max(nrm, 1e-300))
