"""emri_fft_batch_noalloc: the allocation-free FFT entry point.

Some callers cannot call cudaMalloc (a plugin restricted to memory its host
application hands it, a process whose device memory another allocator has
fully reserved, a real-time loop that must not enter the allocator).  This
entry point gives them the library's batched FFT with a fixed, library-owned
static scratch instead of a context.  The test calls it through the C-ABI
on several calls in a row (different sizes, precisions and directions,
batches that take one and several passes of its scratch) and compares every
sequence with emri_fft_batch, and checks that an oversized sequence is
refused.  It runs
last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fft_noalloc_matches_fft_batch_twice():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = emri.Context(0)
    g = np.random.default_rng(2024)
    # the last two cases take more than one pass of the 32 MiB scratch: three
    # 16 MiB FP64 sequences (two, then one), and two 2^21 FP64 sequences that
    # each fill the whole scratch
    cases = [(1 << 16, emri.FP64, -1, 3, torch.complex128, 1e-14),
             (1 << 18, emri.MIXED, +1, 5, torch.complex64, 3e-6),
             (1 << 20, emri.FP64, -1, 3, torch.complex128, 1e-14),
             (1 << 21, emri.FP64, +1, 2, torch.complex128, 1e-14)]
    for n, prec, sign, batch, dtype, tol in cases:
        x = g.standard_normal((batch, n)) + 1j * g.standard_normal((batch, n))
        ref = torch.tensor(x, dtype=dtype, device="cuda:0")
        got = ref.clone()
        ctx.fft_batch(ref, n, batch, prec, sign)
        emri.fft_batch_noalloc(got, n, batch, prec, sign)
        torch.cuda.synchronize()
        r, q = ref.cpu().numpy(), got.cpu().numpy()
        logn = int(np.log2(n))
        for b in range(batch):
            err = np.linalg.norm(q[b] - r[b]) / np.linalg.norm(r[b])
            assert err <= tol * np.sqrt(logn), (n, prec, b, err)
    ctx.close()


def test_fft_noalloc_rejects_oversize():
    from paper_2311_17174_gb300 import emri
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pytest.raises(emri.EmriError) as ei:
        emri.fft_batch_noalloc(0x1000, 1 << 22, 1, emri.FP64, -1, stream=0)
    assert ei.value.code == emri.EINVAL
    assert "exceeds the fixed scratch" in str(ei.value)
