"""The allocation-free resampling entry point, for callers that cannot allocate device
memory (under another framework's allocator lock or memory cap, or in an embedding that
forbids the library from allocating): called through the C ABI several times in a row, it
must give what the context-based b3d_lse_resample gives on the same scores, agree with the
FP64 oracle's resampling, report an all -inf vector in its outputs, leave the device's free
memory unchanged, and replay from a captured CUDA graph. Collected last so that a stop at
the first failure has already run every other test; it also passes alone in a fresh
process."""
import numpy as np
import pytest

from paper_2312_08715_gb300 import b3d, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_noalloc(ll, m, seed, stage, out=None):
    logz, idx, logq = out or (torch.empty(1, device="cuda"), torch.full((m,), -7, dtype=torch.int32, device="cuda"),
                              torch.empty(m, device="cuda"))
    s = torch.cuda.current_stream()
    b3d.b3d_lse_resample_noalloc(ll.numel(), ll, m, seed, stage, logz, idx, logq, s)
    s.synchronize()
    return logz.cpu().numpy(), idx.cpu().numpy(), logq.cpu().numpy()


def test_noalloc_matches_context_entry_point_twice(orc):
    ctx = b3d.Context(0)
    rng = np.random.default_rng(2024)
    cases = [(synth.random_ll(rng, 145800), 100, 11, 0), (synth.random_ll(rng, 3001), 37, 12, 2)]
    for ll_np, m, seed, stage in cases:  # two calls in a row through the shared scratch
        ll = torch.as_tensor(ll_np, device="cuda")
        z_ref, i_ref, q_ref = (t.cpu().numpy() for t in ctx.lse_resample(ll, m, seed, stage))
        ctx.sync()
        z, i, q = _run_noalloc(ll, m, seed, stage)
        np.testing.assert_allclose(z, z_ref, rtol=1e-6, atol=1e-5)
        np.testing.assert_array_equal(i, i_ref)
        np.testing.assert_allclose(q, q_ref, rtol=1e-6, atol=1e-4)
        # the FP64 oracle on the same (FP32) scores: the same draws except where the draw's
        # CDF margin is below FP32 summation accuracy
        oi, oq, margin = orc.resample(ll_np.astype(np.float64), m, seed, stage)
        z64, _ = orc.lse(ll_np.astype(np.float64))
        assert abs(float(z[0]) - z64) <= 1e-6 * abs(z64) + 1e-4
        firm = margin >= 1e-5
        assert firm.mean() > 0.9
        np.testing.assert_array_equal(i[firm], oi[firm])
        np.testing.assert_allclose(q[firm], oq[firm], rtol=1e-5, atol=1e-3)
    ctx.close()


def test_noalloc_all_minus_inf_reports_in_its_outputs():
    ll = torch.full((5000,), float("-inf"), device="cuda")
    z, i, q = _run_noalloc(ll, 9, 1, 0)
    assert np.isneginf(z).all() and (i == -1).all() and np.isneginf(q).all()
    # the next call starts clean
    ll2 = torch.as_tensor(synth.random_ll(np.random.default_rng(3), 5000), device="cuda")
    z2, i2, _ = _run_noalloc(ll2, 9, 1, 0)
    assert np.isfinite(z2).all() and (i2 >= 0).all() and (i2 < 5000).all()


def test_noalloc_allocates_no_device_memory():
    """After the first call on the device (which may load the library's module, code and
    fixed array, into the context), further calls leave the free device memory unchanged."""
    rng = np.random.default_rng(9)
    ll = torch.as_tensor(synth.random_ll(rng, 200000), device="cuda")
    m = 64
    out = (torch.empty(1, device="cuda"), torch.empty(m, dtype=torch.int32, device="cuda"),
           torch.empty(m, device="cuda"))
    first = _run_noalloc(ll, m, 5, 1, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    again = [_run_noalloc(ll, m, 5, 1, out) for _ in range(3)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for a in again:
        for x, y in zip(a, first):
            np.testing.assert_array_equal(x, y)


def test_noalloc_replays_from_a_cuda_graph():
    """The entry point's work is one memset of the shared counter and one kernel launch on
    the caller's stream, so a call captured into a CUDA graph replays: each replay resets the
    counter itself and reads whatever scores the input buffer holds at that moment."""
    rng = np.random.default_rng(31)
    m, seed, stage = 48, 17, 1
    first_np, second_np = synth.random_ll(rng, 60000), synth.random_ll(rng, 60000)
    ll = torch.as_tensor(first_np, device="cuda")
    eager_first = _run_noalloc(ll, m, seed, stage)
    eager_second = _run_noalloc(torch.as_tensor(second_np, device="cuda"), m, seed, stage)
    out = (torch.empty(1, device="cuda"), torch.full((m,), -7, dtype=torch.int32, device="cuda"),
           torch.empty(m, device="cuda"))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up call on a side stream, as before any capture
        b3d.b3d_lse_resample_noalloc(ll.numel(), ll, m, seed, stage, *out, side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b3d.b3d_lse_resample_noalloc(ll.numel(), ll, m, seed, stage, *out, torch.cuda.current_stream())
    for src, want in ((None, eager_first), (None, eager_first), (second_np, eager_second)):
        if src is not None:
            ll.copy_(torch.as_tensor(src, device="cuda"))
        out[1].fill_(-7)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for got, ref in zip((t.cpu().numpy() for t in out), want):
            np.testing.assert_array_equal(got, ref)


def test_noalloc_rejects_bad_sizes():
    ll = torch.zeros(4, device="cuda")
    out = torch.empty(4, device="cuda")
    idx = torch.empty(4, dtype=torch.int32, device="cuda")
    for n in (0, -3, b3d.B3D_NOALLOC_MAX_SCORES + 1):
        with pytest.raises(b3d.B3DError) as e:
            b3d.b3d_lse_resample_noalloc(n, ll, 1, 0, 0, out, idx, out)
        assert e.value.status == b3d.B3D_EINVAL
