"""The allocation-free resampling entry point, for callers that cannot allocate device
memory (e.g. while a CUDA graph is being captured, or under another framework's allocator
lock): called through the C ABI twice in a row, it must give what the context-based
b3d_lse_resample gives on the same scores. Collected last so that a stop at the first
failure has already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2312_08715_gb300 import b3d, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_noalloc(ll, m, seed, stage):
    logz = torch.empty(1, device="cuda")
    idx = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    logq = torch.empty(m, device="cuda")
    s = torch.cuda.current_stream()
    b3d.b3d_lse_resample_noalloc(ll.numel(), ll, m, seed, stage, logz, idx, logq, s)
    s.synchronize()
    return logz.cpu().numpy(), idx.cpu().numpy(), logq.cpu().numpy()


def test_noalloc_matches_context_entry_point_twice():
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
    ctx.close()


def test_noalloc_rejects_bad_sizes():
    ll = torch.zeros(4, device="cuda")
    out = torch.empty(4, device="cuda")
    idx = torch.empty(4, dtype=torch.int32, device="cuda")
    for n in (0, -3, b3d.B3D_NOALLOC_MAX_SCORES + 1):
        with pytest.raises(b3d.B3DError) as e:
            b3d.b3d_lse_resample_noalloc(n, ll, 1, 0, 0, out, idx, out)
        assert e.value.status == b3d.B3D_EINVAL
