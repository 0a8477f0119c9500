"""The learned warm start and block-preconditioner correction on the GPU
(tcgen05 BF16 forward, FP32 backward, Adam, solver integration) against the
FP64 oracle of oracle/mlp.py.

Tolerances: the GPU forward rounds weights and activations to BF16 (8
mantissa bits) with FP32 accumulation; the oracle computes in FP64 with the
same BF16-rounded weights, so outputs and gradients agree to about 1e-2
relative (the bar stated for BF16 outputs)."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2103_01843_gb300.synth import make_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_01843_gb300 as pkg
    pkg.lib()
    return pkg, torch


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), as float64."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _random_params(rng, scale_last=0.05):
    params = omlp.init_params(rng)
    W3, b3 = params[-1]
    params[-1] = (rng.standard_normal(W3.shape) * scale_last, rng.standard_normal(b3.shape) * scale_last)
    return params


def _spd(rng, n):
    A = rng.standard_normal((n, 9, 9))
    D = np.exp(rng.uniform(-2, 5, size=(n, 9)))
    return np.einsum("nij,nkj->nik", A, A) + np.einsum("ni,ij->nij", D, np.eye(9))


def _dev(torch, a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def _bf16_params(params):
    return [(_bf16(W), np.asarray(b, np.float64)) for W, b in params]


@pytest.mark.parametrize("n", [1, 127, 300])
def test_mlp_forward_matches_oracle(env, n):
    pkg, torch = env
    rng = np.random.default_rng(n)
    params = _random_params(rng, 0.2)
    X = rng.standard_normal((n, 19))
    with pkg.Mlp(pkg.mlp_params_flat(params)) as m:
        out = torch.zeros((n, 54), dtype=torch.float32, device="cuda")
        m.forward(_dev(torch, X), out)
        y = out.cpu().numpy().astype(np.float64)
    ref, _ = omlp.forward(_bf16_params(params), _bf16(X))
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= 1e-2, err
    assert np.abs(y - ref).max() <= 3e-2 * np.abs(ref).max()


def test_untrained_output_is_exactly_zero(env):
    pkg, torch = env
    params = omlp.init_params(np.random.default_rng(1))
    with pkg.Mlp(pkg.mlp_params_flat(params)) as m:
        out = torch.full((200, 54), 7.0, dtype=torch.float32, device="cuda")
        m.forward(_dev(torch, np.random.default_rng(2).standard_normal((200, 19))), out)
        assert torch.count_nonzero(out).item() == 0


def test_prepare_matches_oracle(env):
    pkg, torch = env
    rng = np.random.default_rng(3)
    n = 70
    M = _spd(rng, n)
    g = rng.standard_normal((n, 9))
    xs = rng.standard_normal((n, 9))
    cnt = rng.integers(1, 500, n)
    M[5] = -np.eye(9)  # not positive definite: zero features and head inputs
    f_ref, L, w, s, zs = omlp.training_sample(np.where(np.arange(n)[:, None, None] == 5, np.eye(9), M), g, xs, cnt)
    with pkg.Mlp(pkg.mlp_params_flat(omlp.init_params(rng))) as m:
        feats = torch.zeros((n, 19), dtype=torch.float32, device="cuda")
        aux = torch.zeros((n, 72), dtype=torch.float32, device="cuda")
        m.prepare(_dev(torch, M.reshape(n, 81)), _dev(torch, g), _dev(torch, xs),
                  _dev(torch, cnt, torch.int32), feats, aux)
        f, a = feats.cpu().numpy(), aux.cpu().numpy()
    ok = np.arange(n) != 5
    np.testing.assert_allclose(f[ok], f_ref[ok], rtol=2e-4, atol=2e-4)
    tril = np.stack([L[:, i, j] for i in range(9) for j in range(i + 1)], axis=1)
    ref_aux = np.concatenate([tril, w, s, zs], axis=1)
    scale = np.abs(ref_aux[ok]).max(axis=1, keepdims=True)
    assert np.all(np.abs(a[ok] - ref_aux[ok]) <= 1e-4 * scale)
    assert np.all(f[5] == 0) and np.all(a[5] == 0)


def test_loss_and_gradients_match_oracle(env):
    pkg, torch = env
    rng = np.random.default_rng(4)
    n = 333
    params = _random_params(rng, 0.05)
    M = _spd(rng, n)
    g = rng.standard_normal((n, 9))
    xs = np.linalg.solve(M, g[..., None])[..., 0] * (1 + 0.3 * rng.standard_normal((n, 9)))
    X, L, w, s, zs = omlp.training_sample(M, g, xs, rng.integers(1, 100, n))
    aux = np.concatenate([np.stack([L[:, i, j] for i in range(9) for j in range(i + 1)], 1), w, s, zs], 1)
    with pkg.Mlp(pkg.mlp_params_flat(params)) as m:
        loss, grads = m.loss_grad(_dev(torch, X), _dev(torch, aux))
    ref_loss, ref_grads = omlp.loss_and_grads(_bf16_params(params), _bf16(X), L, w, s, zs)
    assert abs(loss - ref_loss) <= 1e-2 * abs(ref_loss)
    got = pkg.mlp_params_unflat(grads)
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(got, ref_grads)):
        eW = np.linalg.norm(gW - rW) / np.linalg.norm(rW)
        eb = np.linalg.norm(gb - rb) / np.linalg.norm(rb)
        assert eW <= 2e-2 and eb <= 2e-2, (li, eW, eb)


def test_training_reduces_loss(env):
    pkg, torch = env
    rng = np.random.default_rng(5)
    n = 1024
    M = _spd(rng, n)
    g = rng.standard_normal((n, 9))
    # a target the untrained model (plain block Jacobi) misses systematically
    xs = np.linalg.solve(M, g[..., None])[..., 0] * 1.5
    X, L, w, s, zs = omlp.training_sample(M, g, xs, np.full(n, 10))
    aux = np.concatenate([np.stack([L[:, i, j] for i in range(9) for j in range(i + 1)], 1), w, s, zs], 1)
    with pkg.Mlp(pkg.mlp_params_flat(omlp.init_params(rng))) as m:
        fx, fa = _dev(torch, X), _dev(torch, aux)
        first = m.train_step(fx, fa, 1e-3)
        for _ in range(200):
            last = m.train_step(fx, fa, 1e-3)
        final, _ = m.loss_grad(fx, fa, with_grads=False)
        prm = m.params()
    assert final < 0.5 * first, (first, last, final)
    assert np.all(np.isfinite(prm))


def test_untrained_model_solves_like_plain(env):
    pkg, torch = env
    s = make_scene("tiny", 0)
    with pkg.Problem.from_scene(s, max_lm_iters=20) as p:
        plain = p.solve()
    model = pkg.Mlp(pkg.mlp_params_flat(omlp.init_params(np.random.default_rng(6))))
    with pkg.Problem.from_scene(s, max_lm_iters=20, use_learned=1) as p:
        p.set_learned(model)
        reps = p.solve()
        assert p.learned_fallbacks() == 0
    f_plain = [r["new_cost"] for r in plain if r["accepted"]][-1]
    f_l = [r["new_cost"] for r in reps if r["accepted"]][-1]
    assert abs(f_plain - f_l) <= 1e-3 * f_plain
    model.close()


def test_learned_requires_a_model_and_single_problems(env):
    pkg, torch = env
    s = make_scene("tiny", 0)
    with pkg.Problem.from_scene(s, use_learned=1) as p:
        p.linearize()
        p.marginalize_qr(1e-4)
        with pytest.raises(pkg.BAError) as e:
            p.pcg_solve()
        assert e.value.status == 4


def test_bad_warm_start_is_dropped(env):
    """A hand-made model whose warm start is no better than the zero start
    (tanh(o) = -1, so x0 = 0 and Q(x0) = 0): the true residual judges it,
    the CG starts from zero and the result equals the plain solve."""
    pkg, torch = env
    params = omlp.init_params(np.random.default_rng(7))
    W3, b3 = params[-1]
    b3 = b3.copy()
    b3[:9] = -20.0
    params[-1] = (W3, b3)
    s = make_scene("tiny", 0)
    with pkg.Problem.from_scene(s) as p:
        p.linearize()
        p.marginalize_qr(1e-4)
        r0 = p.pcg_solve()
        dp0, _ = p.export_step()
    with pkg.Mlp(pkg.mlp_params_flat(params)) as model:
        with pkg.Problem.from_scene(s, use_learned=1) as p:
            p.set_learned(model)
            p.linearize()
            p.marginalize_qr(1e-4)
            r1 = p.pcg_solve()
            dp1, _ = p.export_step()
    assert r1["learned"] == 1 and r1["warm_start"] == 0
    assert np.linalg.norm(dp1 - dp0) <= 1e-3 * np.linalg.norm(dp0)
