"""The allocation-free energy entry point (ba_eval_cost_noalloc) against the
regular one (ba_eval_cost) and the FP64 oracle.

ba_eval_cost_noalloc serves callers that cannot allocate device memory -
latency-critical loops where an allocation would synchronise the device,
programs whose memory belongs to another allocator - by keeping its scratch
in a fixed array inside the library.  This file is collected last so that a
failure here cannot stop the other tests from running first.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2103_01843_gb300.synth import make_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_01843_gb300 as pkg
    pkg.lib()
    return torch, pkg


@pytest.mark.parametrize("name,kw", [("tiny", {}), ("small", dict(n_cam=40, n_pt=30000, p=0.3, cap=40))])
def test_noalloc_cost_matches_eval_cost_on_two_calls(env, name, kw):
    torch, pkg = env
    s = make_scene(name, 2, **kw)
    with pkg.Problem.from_scene(s) as p:
        ref = p.eval_cost()
    dev = torch.device("cuda", torch.cuda.current_device())
    cams = torch.tensor(s.cams.astype(np.float32), device=dev)
    pts = torch.tensor(s.pts.astype(np.float32), device=dev)
    oc = torch.tensor(s.obs_cam, dtype=torch.int32, device=dev)
    op = torch.tensor(s.obs_pt, dtype=torch.int32, device=dev)
    xy = torch.tensor(s.obs_xy.astype(np.float32), device=dev)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    # the oracle's FP64 energy at the FP32-rounded state and observations
    s32 = dataclasses.replace(s, cams=s.cams.astype(np.float32).astype(np.float64),
                              pts=s.pts.astype(np.float32).astype(np.float64),
                              obs_xy=s.obs_xy.astype(np.float32).astype(np.float64))
    e_oracle = oracle.cost(s32)
    for _ in range(2):
        out.fill_(-1.0)
        pkg.eval_cost_noalloc(cams, pts, oc, op, xy, out, stream=stream.cuda_stream)
        stream.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-6 * ref, (got, ref)
        assert abs(got - e_oracle) <= 1e-5 * e_oracle, (got, e_oracle)


def test_noalloc_index_out_of_range_gives_nan(env):
    """An observation whose camera index is n_cam: the result is NaN and no
    out-of-range access is made (the kernel checks the index before loading)."""
    torch, pkg = env
    s = make_scene("tiny", 3)
    dev = torch.device("cuda", torch.cuda.current_device())
    oc_bad = s.obs_cam.copy()
    oc_bad[17] = s.n_cam
    args = [torch.tensor(a, device=dev) for a in (s.cams.astype(np.float32), s.pts.astype(np.float32))]
    oc = torch.tensor(oc_bad, dtype=torch.int32, device=dev)
    op = torch.tensor(s.obs_pt, dtype=torch.int32, device=dev)
    xy = torch.tensor(s.obs_xy.astype(np.float32), device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    pkg.eval_cost_noalloc(args[0], args[1], oc, op, xy, out, stream=stream.cuda_stream)
    stream.synchronize()
    assert np.isnan(float(out.item()))
    # the next valid call is unaffected
    oc = torch.tensor(s.obs_cam, dtype=torch.int32, device=dev)
    pkg.eval_cost_noalloc(args[0], args[1], oc, op, xy, out, stream=stream.cuda_stream)
    stream.synchronize()
    assert np.isfinite(float(out.item()))


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, pkg = env
    dev = torch.device("cuda", torch.cuda.current_device())
    dummy = torch.zeros(16, dtype=torch.float32, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(pkg.BAError) as e:
        pkg.eval_cost_noalloc(dummy, dummy, dummy, dummy, dummy, out, n_cam=1, n_pt=1,
                              n_obs=16384 * 1024 + 1)
    assert e.value.status == 1 and "16777216" in str(e.value)
