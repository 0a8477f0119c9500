"""Parity of the implicit storage (implicit_blocks = 1) with the FP64 oracle.

The implicit form keeps each landmark's factorisation (the pose Jacobian rows,
the Householder vectors and their compact-WY factor, the effect of the damping
rotations) instead of Q2^T J_p and forms the products with A_j on the fly
(the O(k) storage alternative discussed with Table tab:complexities).  It
computes the same reduced camera system (Eq. red_H / red_b) up to rounding, so
it is held to the same bounds as the stored form: reduced system and
preconditioner 1e-4 relative Frobenius, back substitution 1e-4, final LM cost
1e-3 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2103_01843_gb300.synth import degenerate_scene, make_scene
from test_gpu_parity import Rounded, _final, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_01843_gb300 as pkg
    pkg.lib()
    return pkg


SCENES = {
    "tiny": lambda: make_scene("tiny", 0),
    # k up to 100: warp-per-landmark tasks of the implicit matvec (k > 32)
    "heavy": lambda: make_scene("small", 7, n_cam=120, n_pt=600, p=0.05, cap=100),
    # every k from 2 to 32 in one scene: every team width
    "mixed": lambda: make_scene("small", 11, n_cam=40, n_pt=1200, p=0.12, cap=40),
}


@pytest.fixture(scope="module", params=list(SCENES))
def scene(request):
    return request.param, SCENES[request.param]()


def test_reduced_system_and_preconditioner(pkg, scene):
    name, sc = scene
    s = Rounded(sc)
    with pkg.Problem.from_scene(sc, implicit_blocks=1) as p:
        p.linearize()
        for lam in (1e-4, 1e-1, 3e-3):  # re-damping starts from the undamped top rows
            p.marginalize_qr(lam)
            rep = p.pcg_solve()
            M, g = p.export_rcs_diag()
            V = np.random.default_rng(1).normal(size=(3, 9 * s.n_cam)).astype(np.float32)
            Y = np.stack([p.matvec(v) for v in V])
            H_ref, bt_ref = oracle.rcs_dense(s, lam)
            assert rel_fro(Y, V.astype(np.float64) @ H_ref.T) < 1e-4, (name, lam, rel_fro(Y, V @ H_ref.T))
            assert rel_fro(g.ravel(), -bt_ref) < 1e-4, (name, lam)
            Mref = np.stack([H_ref[9 * i:9 * i + 9, 9 * i:9 * i + 9] for i in range(s.n_cam)])
            assert rel_fro(M, Mref) < 1e-4, (name, lam, rel_fro(M, Mref))
            assert rep["precond_fallbacks"] == 0


def test_implicit_equals_stored_blocks(pkg, scene):
    """Same products and blocks as the stored form on the same problem."""
    _, sc = scene
    lam = 2e-3
    out = []
    for imp in (0, 1):
        with pkg.Problem.from_scene(sc, implicit_blocks=imp) as p:
            p.linearize()
            p.marginalize_qr(lam)
            p.pcg_solve()
            M, g = p.export_rcs_diag()
            v = np.random.default_rng(2).normal(size=9 * sc.n_cam).astype(np.float32)
            out.append((p.matvec(v), M, g))
    for a, b in zip(out[0], out[1]):
        assert rel_fro(b, a) < 1e-4


def test_back_substitution_and_solve(pkg):
    tiny = make_scene("tiny", 0)
    s = Rounded(tiny)
    lam = 1e-3
    opt = pkg.default_options(cg_eta=1e-6, implicit_blocks=1)
    ref = oracle.linear_step(s, lam, dense=True)
    with pkg.Problem.from_scene(tiny, options=opt) as p:
        p.linearize()
        p.marginalize_qr(lam)
        p.pcg_solve()
        model = p.backsubstitute()
        dp, dl = p.export_step()
    H_ref, _ = oracle.rcs_dense(s, lam)
    e = dp.ravel().astype(np.float64) - ref["dp"].ravel()
    x = ref["dp"].ravel()
    assert np.sqrt(e @ H_ref @ e) <= 1e-2 * np.sqrt(x @ H_ref @ x)
    dl_ref, model_ref = oracle.backsub_given(s, lam, dp.astype(np.float64))
    assert rel_fro(dl, dl_ref) < 1e-4, rel_fro(dl, dl_ref)
    E = oracle.cost(s)
    assert abs((E - model) - (E - model_ref)) <= 1e-4 * (E - model_ref)


@pytest.mark.parametrize("name", ["tiny", "heavy"])
def test_lm_matches_oracle(pkg, name):
    sc = SCENES[name]()
    s = Rounded(sc)
    iters = 20 if name == "tiny" else 15
    _, _, ref = oracle.lm(s, max_iters=iters, dense=False)
    with pkg.Problem.from_scene(sc, max_lm_iters=iters, implicit_blocks=1) as p:
        reps = p.solve()
    assert abs(_final(reps) - _final(ref)) <= 1e-3 * _final(ref), (_final(reps), _final(ref))
    n = min(3, len(reps), len(ref))
    assert [r["accepted"] for r in reps[:n]] == [int(e["accepted"]) for e in ref[:n]]


@pytest.mark.parametrize("lam", [1e-4, 1e-8])
def test_degenerate_landmarks(pkg, lam):
    """A zero depth column, a single-centre landmark and one at 0.08 m depth:
    the implicit products equal the oracle's; camera 8's block would cancel in
    the Gram form and is summed from the factorisation instead."""
    sc, sp = degenerate_scene(0)
    s = Rounded(sc)
    with pkg.Problem.from_scene(sc, implicit_blocks=1) as p:
        p.linearize()
        p.marginalize_qr(lam)
        rep = p.pcg_solve()
        M, g = p.export_rcs_diag()
        V = np.random.default_rng(4).normal(size=(3, 9 * s.n_cam)).astype(np.float32)
        Y = np.stack([p.matvec(v) for v in V])
    H_ref, bt_ref = oracle.rcs_dense(s, lam)
    assert rel_fro(Y, V.astype(np.float64) @ H_ref.T) < 1e-4
    assert rel_fro(g.ravel(), -bt_ref) < 1e-4
    for i in range(s.n_cam):
        assert rel_fro(M[i], H_ref[9 * i:9 * i + 9, 9 * i:9 * i + 9]) < 1e-4, i
    assert rep["precond_exact"] >= 1 and rep["precond_fallbacks"] == 0


def test_blocks_from_the_factorisation_for_every_camera(pkg):
    """precond_from_blocks = 1 with implicit storage: every camera's block and
    g are summed from the factorisation (no Gram identity)."""
    sc = SCENES["heavy"]()
    s = Rounded(sc)
    lam = 1e-2
    with pkg.Problem.from_scene(sc, implicit_blocks=1, precond_from_blocks=1) as p:
        p.linearize()
        p.marginalize_qr(lam)
        rep = p.pcg_solve()
        M, g = p.export_rcs_diag()
    Mref, bt = oracle.rcs_diag(s, lam)
    assert rel_fro(M, Mref) < 1e-4 and rel_fro(g, -bt) < 1e-4
    assert rep["precond_exact"] == s.n_cam


def test_long_tracks(pkg):
    """Tracks of up to 300 observations (ten chunks of one warp)."""
    sc = make_scene("small", 13, n_cam=320, n_pt=60, p=0.005, cap=300)
    s = Rounded(sc)
    lam = 1e-3
    with pkg.Problem.from_scene(sc, implicit_blocks=1) as p:
        p.linearize()
        p.marginalize_qr(lam)
        p.pcg_solve()
        M, g = p.export_rcs_diag()
        V = np.random.default_rng(9).normal(size=(2, 9 * s.n_cam)).astype(np.float32)
        Y = np.stack([p.matvec(v) for v in V])
    Mref, bt = oracle.rcs_diag(s, lam)
    assert rel_fro(M, Mref) < 1e-4
    assert rel_fro(g, -bt) < 1e-4
    assert rel_fro(Y, oracle.rcs_matvec(s, lam, V)) < 1e-4


def test_many_cameras_y_in_global_memory(pkg):
    """6000 cameras: y (9 n_cam floats) no longer fits the matvec's shared
    memory and is accumulated in global memory."""
    sc = make_scene("small", 17, n_cam=6000, n_pt=3000, p=0.3, cap=12)
    s = Rounded(sc)
    lam = 1e-3
    with pkg.Problem.from_scene(sc, implicit_blocks=1) as p:
        p.linearize()
        p.marginalize_qr(lam)
        V = np.random.default_rng(3).normal(size=(2, 9 * s.n_cam)).astype(np.float32)
        Y = np.stack([p.matvec(v) for v in V])
    assert rel_fro(Y, oracle.rcs_matvec(s, lam, V)) < 1e-4


def test_rebuilt_top_rows_match_the_stored_form(pkg, scene):
    """The implicit storage keeps no top rows [Q1^T J_p | R1 | Q1^T r]; the
    export rebuilds them from the records (D_s - P V_s^T J_s, R1, Q1^T r),
    the way K3 and the back substitution do.  Against the stored form's rows
    (the same Householder reflections), undamped, on landmarks of every k."""
    name, sc = scene
    with pkg.Problem.from_scene(sc, implicit_blocks=1) as p, pkg.Problem.from_scene(sc) as q:
        p.linearize()
        q.linearize()
        ks = np.bincount(sc.obs_pt, minlength=sc.n_pt)  # observations per landmark
        js = sorted({int(np.argmax(ks))} | {int(np.flatnonzero(ks == k)[0]) for k in np.unique(ks)[:12]})
        for j in js:
            a = p.export_landmark(j, k_cap=int(ks.max()), top_only=True)["top"]
            b = q.export_landmark(j, k_cap=int(ks.max()))["top"]
            assert a.shape == b.shape and a.size == 3 * (9 * ks[j] + 4)
            assert rel_fro(a, b) < 1e-5, (name, j, int(ks[j]), rel_fro(a, b))


def test_option_is_fixed_at_create(pkg):
    tiny = make_scene("tiny", 0)
    with pkg.Problem.from_scene(tiny, implicit_blocks=1) as p:
        with pytest.raises(pkg.BAError) as e:
            p.set_options(implicit_blocks=0)
        assert e.value.status == 1
        p.linearize()
        with pytest.raises(pkg.BAError):
            p.export_landmark(0)
        top = p.export_landmark(0, top_only=True)["top"]
        assert np.isfinite(top).all()
    with pytest.raises(pkg.BAError):
        pkg.Problem.from_scene(tiny, implicit_blocks=2)


def test_batch_with_implicit_storage(pkg):
    """A batch of uneven problems in the implicit storage: every member's
    final cost against the oracle's LM on that member alone."""
    members = [make_scene("batched_member", s) for s in (0, 1)]
    members.append(SCENES["heavy"]())
    iters = 10
    with pkg.Batch(members, max_lm_iters=iters, implicit_blocks=1) as b:
        reps, _ = b.solve()
    for s, r in zip(members, reps):
        _, _, log = oracle.lm(Rounded(s), max_iters=iters, dense=False)
        ref = _final(log)
        assert abs(r["final_cost"] - ref) <= 1e-3 * ref, (r, ref)
