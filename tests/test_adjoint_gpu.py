"""Receptor concentrations and the hand-written adjoint on the GPU, through the C ABI and
the torch.autograd.Function: against the oracle on the same particles, against central
finite differences of the GPU forward with the same seeds, against the analytic plume
gradient in the uniform-weather setting, and for the exact structure in q."""
import dataclasses
import math

import numpy as np
import pytest

import lpm_inputs as li
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIGMA = 200.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0912_3223_gb300 import build
    build.build()
    oracle.build()


def _sim(cfg):
    from paper_0912_3223_gb300 import Sim
    return Sim(cfg)


def _uniform(n, steps, q=None):
    cfg = li.make_cfg0(n_particles=n, n_steps=steps)
    if q is not None:
        cfg = dataclasses.replace(cfg, release=dataclasses.replace(cfg.release, q=np.asarray(q),
                                                                    q_dt=300.0))
    return cfg


REC0 = np.array([[2000.0, 0.0, 2.0], [2500.0, 300.0, 10.0], [1500.0, -200.0, 40.0],
                 [3000.0, 150.0, 80.0]])
W0 = np.array([1.0, -0.5, 2.0, 0.7])


def _realistic(n=3000, steps=360):
    cfg = li.make_cfg3(n_particles=n, n_steps=steps)
    rec = li.make_receptors()
    return cfg, rec


def test_receptors_match_oracle():
    from paper_0912_3223_gb300 import lpm
    for cfg, rec in [(_uniform(3000, 120, q=[1.0, 2.0, 0.5, 1.5]), REC0), _realistic()]:
        with _sim(cfg) as sim:
            C = lpm.lpm_receptors(sim.ctx, 1, rec, SIGMA, 12)[0]
        ref = oracle.receptors(cfg, rec, SIGMA, 12)
        scale = np.abs(ref).max()
        assert scale > 0
        np.testing.assert_allclose(C, ref, rtol=1e-3, atol=1e-4 * scale)


def test_adjoint_matches_oracle_uniform_weather():
    from paper_0912_3223_gb300 import lpm
    cfg = _uniform(3000, 120, q=[1.0, 2.0, 0.5, 1.5])
    with _sim(cfg) as sim:
        g = lpm.lpm_adjoint(sim.ctx, REC0, SIGMA, 10, W0[None, :], 4)[0]
    ref = oracle.adjoint(cfg, REC0, SIGMA, 10, W0)
    np.testing.assert_allclose(g, ref, rtol=1e-3, atol=1e-4 * np.abs(ref).max())


def test_adjoint_matches_oracle_realistic_weather():
    """Sheared, height-dependent weather with decay and deposition (events frozen): FP32
    pathwise gradients follow the FP64 ones; the bar is 1 % of the largest component
    (chaotic near-ground paths carry most of the difference)."""
    from paper_0912_3223_gb300 import lpm
    cfg, rec = _realistic()
    w = np.linspace(-1.0, 1.0, rec.shape[0])
    with _sim(cfg) as sim:
        g = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w[None, :], 24)[0]
    ref = oracle.adjoint(cfg, rec, SIGMA, 18, w)
    src_ref, src = ref[:3], g[:3]
    np.testing.assert_allclose(src, src_ref, atol=0.01 * np.abs(src_ref).max())
    np.testing.assert_allclose(g[3:27], ref[3:27], rtol=1e-3, atol=1e-6 * np.abs(ref[3:27]).max())
    np.testing.assert_allclose(g[27:], ref[27:], atol=0.01 * np.abs(ref[27:]).max())
    assert np.all(g[3 + 6:27] == 0.0)       # emission hours after the 2 h run


def test_adjoint_matches_gpu_central_fd():
    """Central finite differences of the GPU forward with the same seeds."""
    from paper_0912_3223_gb300 import lpm
    cfg = _uniform(4000, 120, q=[1.0, 2.0])
    with _sim(cfg) as sim:
        def L():
            return float(W0 @ lpm.lpm_receptors(sim.ctx, 1, REC0, SIGMA, 10)[0])
        g = lpm.lpm_adjoint(sim.ctx, REC0, SIGMA, 10, W0[None, :], 2)[0]
        h = 0.5
        fd = []
        for d in range(3):
            base = [cfg.src_x, cfg.src_y, cfg.src_z]
            p = list(base); p[d] += h
            m = list(base); m[d] -= h
            lpm.lpm_set_source(sim.ctx, 0, *p)
            lp = L()
            lpm.lpm_set_source(sim.ctx, 0, *m)
            lm = L()
            fd.append((lp - lm) / (2 * h))
        lpm.lpm_set_source(sim.ctx, 0, cfg.src_x, cfg.src_y, cfg.src_z)
        for idx, (a, b) in enumerate([((1.01, 0, 0), (0.99, 0, 0)), ((1, 0.01, 0), (1, -0.01, 0)),
                                      ((1, 0, 0.01), (1, 0, -0.01))]):
            lpm.lpm_set_params(sim.ctx, *a)
            lp = L()
            lpm.lpm_set_params(sim.ctx, *b)
            lm = L()
            fd.append((lp - lm) / 0.02)
        lpm.lpm_set_params(sim.ctx, 1.0, 0.0, 0.0)
    got = np.concatenate([g[:3], g[-3:]])
    fd = np.array(fd)
    np.testing.assert_allclose(got, fd, atol=2e-3 * np.abs(fd).max(), rtol=5e-3)


def test_autograd_function_and_analytic_plume_gradient():
    """torch.autograd.Function on 1e6 particles in the uniform-weather setting: the
    gradient matches the exact gradient of the expected loss within Monte-Carlo error
    (estimated from the spread of 8 independent seeds)."""
    from paper_0912_3223_gb300.adjoint import receptor_concentrations
    from test_oracle_adjoint import _expected_loss
    n, S, every = 1_000_000, 60, 6
    rec = np.array([[900.0, 0.0, 2.0], [1200.0, 250.0, 60.0], [600.0, -150.0, 25.0]])
    w = torch.tensor([1.0, 1.5, -0.8], dtype=torch.float64)
    grads = []
    for seed in range(1, 9):
        cfg = dataclasses.replace(_uniform(n, S), seed=seed)
        with _sim(cfg) as sim:
            src = torch.tensor([[0.0, 0.0, 50.0]], dtype=torch.float64, requires_grad=True)
            q = torch.tensor([[1.0]], dtype=torch.float64, requires_grad=True)
            ks = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
            b = torch.zeros(2, dtype=torch.float64, requires_grad=True)
            C = receptor_concentrations(sim, src, q, ks, b, rec, SIGMA, every)
            (C[0] * w).sum().backward()
            grads.append(np.concatenate([src.grad[0].numpy(), [ks.grad.item()], b.grad.numpy()]))
    grads = np.array(grads)
    mc = grads.mean(0)
    se = grads.std(0, ddof=1) / math.sqrt(len(grads))
    theta = np.array([0.0, 0.0, 50.0, 1.0, 0.0, 0.0])
    cfg = _uniform(n, S)
    exact = []
    for i in range(6):
        hs = 1e-3 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += hs
        tm[i] -= hs
        exact.append((_expected_loss(tp, cfg, every, rec, w.numpy()) -
                      _expected_loss(tm, cfg, every, rec, w.numpy())) / (2 * hs))
    exact = np.array(exact)
    assert np.all(np.abs(mc - exact) < 5 * se + 2e-3 * np.abs(exact).max()), (mc, exact, se)


def test_emission_gradient_is_exactly_linear():
    from paper_0912_3223_gb300 import lpm
    cfg = _uniform(2000, 60, q=[1.0, 2.0, 0.5, 1.5, 3.0])
    with _sim(cfg) as sim:
        g = lpm.lpm_adjoint(sim.ctx, REC0, SIGMA, 6, W0[None, :], 5)[0]
        for hq in range(5):
            e = np.zeros(5)
            e[hq] = 1.0
            lpm.lpm_set_emission(sim.ctx, 0, e)
            L = float(W0 @ lpm.lpm_receptors(sim.ctx, 1, REC0, SIGMA, 6)[0])
            assert g[3 + hq] == pytest.approx(L, rel=2e-5, abs=1e-12 * abs(g).max())
    assert g[3 + 2] == 0.0 and g[3 + 4] == 0.0


def test_batched_inversion_reduces_misfit_and_approaches_the_hidden_source():
    """A small inversion: 8 candidates x 20000 particles, 2 h, 12 Adam iterations against
    observations of a hidden source (independent key): every candidate's misfit drops and
    the best candidate ends closer to the hidden source than the best start."""
    from paper_0912_3223_gb300 import Sim
    from paper_0912_3223_gb300.inversion import invert, observe
    cand, obs, hidden = li.make_cfg4(n_candidates=8, n_per=20_000, n_steps=360, n_obs=100_000)
    rec = li.make_receptors()
    with Sim(obs) as so:
        c_obs = observe(so, rec, 200.0, 18)
    assert c_obs.max() > 0
    with Sim(cand) as sc:
        res = invert(sc, rec, c_obs, n_iter=12)
    start, end = res.loss[0], res.loss[-1]
    print("loss start", np.round(start, 3), "end", np.round(end, 3))
    moved = np.abs(res.grad).sum(axis=(0, 2)) > 0          # candidates that see the plume
    assert moved.any()
    assert np.all(end[moved] <= start[moved] * 1.05)
    assert end.min() < 0.9 * start.min()
    h = np.array(hidden)
    d0 = np.linalg.norm(res.sources[0, :, :2] - h[:2], axis=1)
    d1 = np.linalg.norm(res.sources[-1, :, :2] - h[:2], axis=1)
    print("best candidate distance to the hidden source: start", d0.min(), "end", d1[res.best])
    assert d1[res.best] < d0.min()


def test_trajectory_and_checkpoint_storage_agree():
    """The backward forms take the same paths and events, so receptors and gradients agree
    to the order of the FP64 sums: the trajectory re-sorted by weather cell every 64 steps
    (one scenario, sorting on), the trajectory in release order (sorting off, or a batch of
    candidates), and 64-step checkpoints with recomputation (a limit below the trajectory's
    size), in sorted segments (sorting on) or in release order. One scenario with
    deposition and exits, and a batch of three (sorted by scenario, then cell tile)."""
    from paper_0912_3223_gb300 import Sim, lpm
    cfg, rec = _realistic(n=5000, steps=400)
    cand, _, _ = li.make_cfg4(n_candidates=3, n_per=3000, n_steps=300, n_obs=1000)
    for c, nq in [(cfg, 24), (cand, 24)]:
        w = np.linspace(-1.0, 1.0, c.n_scenarios * rec.shape[0]).reshape(c.n_scenarios, -1)
        out = {}
        for form, limit, sort in [("trajectory", 1 << 37, 60), ("release order", 1 << 37, 0),
                                  ("checkpoints", 0, 60), ("checkpoints (limit)", 1024, 60),
                                  ("checkpoints in release order", 0, 0)]:
            with Sim(c) as sim:
                lpm.lpm_set_sort(sim.ctx, sort)
                lpm.lpm_set_adjoint_storage(sim.ctx, limit)
                C = lpm.lpm_receptors(sim.ctx, c.n_scenarios, rec, SIGMA, 18)
                g = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w, nq)
                g2 = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, 2.0 * w, nq)   # held forward reused
                traj, nbytes = lpm.lpm_adjoint_storage(sim.ctx)
            assert traj == (limit == 1 << 37)
            assert nbytes > 0
            np.testing.assert_allclose(g2, 2.0 * g, rtol=1e-12, atol=1e-15 * np.abs(g).max())
            out[form] = (C, g)
        # same order of the per-particle FP32 sums: agree to the order of the FP64 sums
        C0, g0 = out["release order"]
        assert np.abs(g0).max() > 0
        # the sorted checkpoint form sweeps the same entries in the same order as the
        # sorted trajectory (for a batch: sorted by scenario, then cell tile)
        pairs = [("checkpoints in release order", "release order")]
        pairs += [(f, "trajectory") for f in ("checkpoints", "checkpoints (limit)")]
        for form, base in pairs:
            C1, g1 = out[form]
            Cb, gb = out[base]
            np.testing.assert_allclose(C1, Cb, rtol=1e-12, atol=1e-15 * np.abs(Cb).max(),
                                       err_msg=form)
            np.testing.assert_allclose(g1, gb, rtol=1e-9, atol=1e-12 * np.abs(gb).max(),
                                       err_msg=form)
        # the sorted form carries dL/dX between segments exactly (FP32 values; sums over
        # particles are FP64) but restarts each particle's FP32 parameter sums every 64
        # steps: source partials to the order of the FP64 sums, parameter partials to FP32
        # rounding of the per-particle sums
        C1, g1 = out["trajectory"]
        np.testing.assert_allclose(C1, C0, rtol=1e-12, atol=1e-15 * np.abs(C0).max())
        np.testing.assert_allclose(g1[:, :3], g0[:, :3], rtol=1e-9,
                                   atol=1e-12 * np.abs(g0[:, :3]).max())
        np.testing.assert_allclose(g1[:, 3:], g0[:, 3:], rtol=0,
                                   atol=2e-5 * np.abs(g0[:, 3:]).max())


def test_sorted_trajectory_with_late_release_and_partial_segment_matches_oracle():
    """Segment edges of the cell-sorted form: a release window [70, 380) that starts and ends
    inside 64-step segments, in a 401-step run whose last segment holds 17 steps, against
    the oracle and against the recomputing checkpoint form."""
    from paper_0912_3223_gb300 import Sim, lpm
    cfg, rec = _realistic(n=4000, steps=401)
    cfg = dataclasses.replace(cfg, release=dataclasses.replace(cfg.release, first_step=70,
                                                               last_step=380))
    w = np.linspace(-1.0, 1.0, rec.shape[0])
    out = {}
    for limit in (1 << 37, 0):
        with Sim(cfg) as sim:
            lpm.lpm_set_adjoint_storage(sim.ctx, limit)
            C = lpm.lpm_receptors(sim.ctx, 1, rec, SIGMA, 18)[0]
            g = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w[None, :], 24)[0]
            assert lpm.lpm_adjoint_storage(sim.ctx)[0] == (limit != 0)
        out[limit] = (C, g)
    C, g = out[1 << 37]
    C1, g1 = out[0]
    np.testing.assert_allclose(C1, C, rtol=1e-12, atol=1e-15 * np.abs(C).max())
    np.testing.assert_allclose(g1[:3], g[:3], rtol=1e-9, atol=1e-12 * np.abs(g[:3]).max())
    np.testing.assert_allclose(g1[3:], g[3:], rtol=0, atol=2e-5 * np.abs(g[3:]).max())
    ref_C = oracle.receptors(cfg, rec, SIGMA, 18)
    assert np.abs(ref_C).max() > 0
    np.testing.assert_allclose(C, ref_C, rtol=1e-3, atol=1e-4 * np.abs(ref_C).max())
    ref = oracle.adjoint(cfg, rec, SIGMA, 18, w)
    np.testing.assert_allclose(g[:3], ref[:3], atol=0.01 * np.abs(ref[:3]).max())
    np.testing.assert_allclose(g[3:27], ref[3:27], rtol=1e-3, atol=1e-6 * np.abs(ref[3:27]).max())
    np.testing.assert_allclose(g[27:], ref[27:], atol=0.01 * np.abs(ref[27:]).max())


def test_checkpoint_segments_on_two_streams_match_the_trajectory():
    """The checkpoint form recomputes segment s - 1 on a second stream while segment s is
    swept, the two segments in the two halves of a scratch: runs of one, two, three and
    seven segments (the last one partial) give the sorted trajectory form's receptors and
    gradients, and repeated sweeps of the same held forward give the same gradients."""
    from paper_0912_3223_gb300 import Sim, lpm
    for steps in (50, 128, 150, 401):
        cfg, rec = _realistic(n=2500, steps=steps)
        every = 9
        w = np.linspace(-1.0, 1.0, rec.shape[0])[None, :]
        out = {}
        for limit in (1 << 37, 0):
            with Sim(cfg) as sim:
                lpm.lpm_set_adjoint_storage(sim.ctx, limit)
                C = lpm.lpm_receptors(sim.ctx, 1, rec, SIGMA, every)
                gs = [lpm.lpm_adjoint(sim.ctx, rec, SIGMA, every, w, 24) for _ in range(3)]
                assert lpm.lpm_adjoint_storage(sim.ctx)[0] == (limit != 0)
            for g in gs[1:]:
                np.testing.assert_allclose(g, gs[0], rtol=1e-12, atol=1e-15 * np.abs(gs[0]).max())
            out[limit] = (C, gs[0])
        (C0, g0), (C1, g1) = out[1 << 37], out[0]
        assert np.abs(g0).max() > 0, steps
        np.testing.assert_allclose(C1, C0, rtol=1e-12, atol=1e-15 * np.abs(C0).max(),
                                   err_msg=str(steps))
        np.testing.assert_allclose(g1, g0, rtol=1e-9, atol=1e-12 * np.abs(g0).max(),
                                   err_msg=str(steps))


def test_adjoint_with_gridded_kh_matches_oracle_in_every_storage_form():
    """A gridded K_h field brings its spatial gradient into the transposed Jacobian (the
    sqrt(K_h) derivative of the horizontal displacement): the cell-sorted trajectory, the
    release-order trajectory and the checkpoint forms against the oracle."""
    from paper_0912_3223_gb300 import Sim, lpm
    cfg, rec = _realistic(n=3000, steps=360)
    rng = np.random.default_rng(21)
    kh = (60.0 + 80.0 * rng.random(cfg.uvwk.shape[:-1])).astype(np.float32)
    cfg = dataclasses.replace(cfg, kh=kh, kh_uniform=-1.0)
    w = np.linspace(-1.0, 1.0, rec.shape[0])
    ref = oracle.adjoint(cfg, rec, SIGMA, 18, w)
    assert np.abs(ref[27:28]).max() > 0
    for limit, sort in ((1 << 37, 60), (1 << 37, 0), (0, 60), (0, 0)):
        with Sim(cfg) as sim:
            lpm.lpm_set_sort(sim.ctx, sort)
            lpm.lpm_set_adjoint_storage(sim.ctx, limit)
            g = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w[None, :], 24)[0]
        np.testing.assert_allclose(g[:3], ref[:3], atol=0.01 * np.abs(ref[:3]).max())
        np.testing.assert_allclose(g[3:27], ref[3:27], rtol=1e-3,
                                   atol=1e-6 * np.abs(ref[3:27]).max())
        np.testing.assert_allclose(g[27:], ref[27:], atol=0.01 * np.abs(ref[27:]).max())


def test_batched_adjoint_matches_oracle_per_scenario():
    """The batched adjoint the inversion uses (three candidate sources in one context, one
    launch for all): each scenario's gradient against the oracle's adjoint of that
    scenario alone, with its own dL/dC."""
    from paper_0912_3223_gb300 import Sim, lpm
    cand, _, _ = li.make_cfg4(n_candidates=3, n_per=3000, n_steps=300, n_obs=1000)
    rec = li.make_receptors()
    rng = np.random.default_rng(5)
    w = rng.normal(0.0, 1.0, (cand.n_scenarios, rec.shape[0]))
    with Sim(cand) as sim:
        g = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w, 24)
    seen = 0
    for s in range(cand.n_scenarios):
        ref = oracle.adjoint(cand, rec, SIGMA, 18, w[s], scenario=s)
        if np.abs(ref[:3]).max() == 0:
            assert np.abs(g[s, :3]).max() == 0          # the plume misses every receptor
            continue
        seen += 1
        np.testing.assert_allclose(g[s, :3], ref[:3], atol=0.01 * np.abs(ref[:3]).max())
        np.testing.assert_allclose(g[s, 3:27], ref[3:27], rtol=1e-3,
                                   atol=1e-6 * np.abs(ref[3:27]).max())
        np.testing.assert_allclose(g[s, 27:], ref[27:], atol=0.01 * np.abs(ref[27:]).max())
    assert seen >= 1


def test_sorted_batch_with_many_small_scenarios_matches_release_order_and_oracle():
    """Twenty-four candidates of 230 particles: blocks of 128 sorted entries straddle the
    scenario boundaries, so many entries add their receptor sums and gradients to their own
    scenario's global sums instead of their block's. The sorted trajectory and checkpoint
    forms against the release-order trajectory (source partials to the order of the FP64
    sums; the others to FP32 rounding of the per-segment sums), and two scenarios against
    the oracle."""
    from paper_0912_3223_gb300 import Sim, lpm
    cand, _, _ = li.make_cfg4(n_candidates=24, n_per=230, n_steps=260, n_obs=500)
    rec = li.make_receptors()
    rng = np.random.default_rng(11)
    w = rng.normal(0.0, 1.0, (cand.n_scenarios, rec.shape[0]))
    out = {}
    for form, limit, sort in [("sorted", 1 << 37, 60), ("sorted checkpoints", 0, 60),
                              ("release order", 1 << 37, 0)]:
        with Sim(cand) as sim:
            lpm.lpm_set_sort(sim.ctx, sort)
            lpm.lpm_set_adjoint_storage(sim.ctx, limit)
            C = lpm.lpm_receptors(sim.ctx, cand.n_scenarios, rec, SIGMA, 18)
            g = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w, 24)
        out[form] = (C, g)
    C0, g0 = out["release order"]
    assert np.abs(C0).max() > 0 and np.abs(g0).max() > 0
    for form in ("sorted", "sorted checkpoints"):
        C1, g1 = out[form]
        np.testing.assert_allclose(C1, C0, rtol=1e-12, atol=1e-15 * np.abs(C0).max(), err_msg=form)
        np.testing.assert_allclose(g1[:, :3], g0[:, :3], rtol=1e-9,
                                   atol=1e-12 * np.abs(g0[:, :3]).max(), err_msg=form)
        np.testing.assert_allclose(g1[:, 3:], g0[:, 3:], rtol=0,
                                   atol=2e-5 * np.abs(g0[:, 3:]).max(), err_msg=form)
    np.testing.assert_allclose(out["sorted checkpoints"][1], out["sorted"][1], rtol=1e-9,
                               atol=1e-12 * np.abs(out["sorted"][1]).max())
    g = out["sorted"][1]
    hit = [s for s in range(cand.n_scenarios) if np.abs(g0[s, :3]).max() > 0]
    assert len(hit) >= 2
    for s in hit[:2]:
        ref = oracle.adjoint(cand, rec, SIGMA, 18, w[s], scenario=s)
        np.testing.assert_allclose(g[s, :3], ref[:3], atol=0.01 * np.abs(ref[:3]).max())
        np.testing.assert_allclose(g[s, 3:27], ref[3:27], rtol=1e-3,
                                   atol=1e-6 * np.abs(ref[3:27]).max())


def test_partitioned_receptors_and_adjoint_sum_to_single_context():
    """Three contexts holding disjoint particle ranges of one release, run one after
    another on this GPU as the ranks of a partitioned run would: their receptor sums, and
    their gradients of a misfit whose dL/dC is formed from the summed concentrations, add
    up in fixed point to the single-context values (the per-particle arithmetic is the
    same; only the FP64 summation order differs)."""
    from paper_0912_3223_gb300 import Sim, lpm
    from paper_0912_3223_gb300.parallel import partition, sum_float_fixed
    cfg, rec = _realistic(n=3001, steps=360)
    nq = cfg.release.q.size
    parts_c = []
    for r in range(3):
        with Sim(cfg, part=partition(cfg.n_particles, 3, r)) as sim:
            parts_c.append(lpm.lpm_receptors(sim.ctx, 1, rec, SIGMA, 18))
    c = sum_float_fixed(parts_c)
    w = 2.0 * (c - 0.5 * c)                      # dL/dC of sum (C - C/2)^2
    parts_g = []
    for r in range(3):
        with Sim(cfg, part=partition(cfg.n_particles, 3, r)) as sim:
            parts_g.append(lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w, nq))
    g = sum_float_fixed(parts_g)
    with Sim(cfg) as sim:
        c_full = lpm.lpm_receptors(sim.ctx, 1, rec, SIGMA, 18)
        g_full = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 18, w, nq)
    assert np.abs(c_full).max() > 0 and np.abs(g_full).max() > 0
    dc = np.abs(c - c_full).max() / np.abs(c_full).max()
    dg = np.abs(g - g_full).max() / np.abs(g_full).max()
    print(f"partitioned vs single context: receptors {dc:.2e}, gradient {dg:.2e}")
    np.testing.assert_allclose(c, c_full, rtol=1e-12, atol=1e-14 * np.abs(c_full).max())
    np.testing.assert_allclose(g, g_full, rtol=1e-12, atol=1e-14 * np.abs(g_full).max())


def test_adjoint_at_the_maximum_receptors_and_emission_values():
    """256 receptors and a 64-value emission series, the adjoint's limits: receptor
    concentrations and the gradient against the oracle, emission values after the run with
    a zero gradient; one receptor or one emission value more is rejected on the host."""
    from paper_0912_3223_gb300 import lpm
    rng = np.random.default_rng(21)
    q = np.exp(rng.normal(0.0, 0.3, 64))
    cfg = li.make_cfg0(n_particles=3000, n_steps=120)
    cfg = dataclasses.replace(cfg, release=dataclasses.replace(cfg.release, q=q, q_dt=20.0))
    xs, ys = np.meshgrid(np.linspace(300.0, 4800.0, 16), np.linspace(-750.0, 750.0, 16))
    rec = np.stack([xs.ravel(), ys.ravel(), np.full(256, 10.0)], 1)
    w = rng.normal(size=256)
    with _sim(cfg) as sim:
        C = lpm.lpm_receptors(sim.ctx, 1, rec, SIGMA, 10)[0]
        g = lpm.lpm_adjoint(sim.ctx, rec, SIGMA, 10, w[None, :], 64)[0]
        for bad in (lambda: lpm.lpm_receptors(sim.ctx, 1, np.vstack([rec, rec[:1]]), SIGMA, 10),
                    lambda: lpm.lpm_set_emission(sim.ctx, 0, np.ones(65))):
            with pytest.raises(lpm.LpmError) as e:
                bad()
            assert e.value.status == lpm.LPM_E_INVALID
    ref_c = oracle.receptors(cfg, rec, SIGMA, 10)
    assert np.count_nonzero(ref_c) > 100
    np.testing.assert_allclose(C, ref_c, rtol=1e-3, atol=1e-4 * np.abs(ref_c).max())
    ref = oracle.adjoint(cfg, rec, SIGMA, 10, w)
    np.testing.assert_allclose(g, ref, rtol=1e-3, atol=1e-4 * np.abs(ref).max())
    assert np.all(g[3 + 60:3 + 64] == 0.0)     # 20 s emission bins after the 1200 s run
    assert np.all(g[3:3 + 60] != 0.0)
