"""The VMC moves and the learned proposal on the GPU: the perceptron's forward
and backward kernels and both training objectives against the FP64 reference
in oracle/mlp.py, the proposal densities, the zero-network limit (the
drift-diffusion move), sampler invariance, and the gain of the trained
proposal over plain drift-diffusion in autocorrelation-corrected samples/s."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import mlp as omlp
import paper_1510_00730_gb300 as pkg
from paper_1510_00730_gb300 import binding as B
from paper_1510_00730_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _mlp(n_elec=17, hidden=256, seed=9, langevin=True, zero_head=False, mm=0.8, s0=-2.0, span=1.5, scale=2.0):
    return B.MLP(0, n_elec, hidden=hidden, seed=seed, mu_max=mm, s0=s0, s_span=span, coord_scale=scale,
                 langevin=langevin, zero_head=zero_head)


def test_mlp_forward_matches_oracle():
    """Forward pass on the tcgen05 tensor cores (BF16 weights and activations, FP32
    accumulation) vs the FP64 network with the same BF16 rounding points (acts_bf16).

    Tolerance: an activation within an FP32 rounding error of a BF16 rounding boundary
    may round the other way on the GPU (FP32 tanh and sums) than in the oracle (FP64):
    one BF16 unit, at most 2^-8 |h| <= 2^-8, which moves an output by at most
    2^-8 max|W3| = 2^-8 sqrt(6 / (256 + 68)) = 5.3e-4. So the bound is 1e-3 per output
    (relative above 1), while the bulk of the outputs must agree to FP32 accumulation."""
    m = _mlp()
    rng = np.random.default_rng(1)
    R = rng.normal(scale=1.5, size=(300, 17, 3))
    out = m.forward(_t(R)).cpu().numpy()
    ref, _ = omlp.forward(m.params(), R, 17, 256, 2.0, acts_bf16=True)
    err = np.abs(out - ref) / np.maximum(np.abs(ref), 1.0)
    assert err.max() <= 1e-3, err.max()
    assert np.median(err) <= 1e-5, np.median(err)
    # the rounding points matter: without them the oracle is much farther from the GPU
    plain, _ = omlp.forward(m.params(), R, 17, 256, 2.0, acts_bf16=False)
    assert np.median(np.abs(out - plain) / np.maximum(np.abs(plain), 1.0)) > 10 * np.median(err)
    m.close()


def test_mlp_nll_gradient_matches_oracle():
    """NLL loss, dL/d(out) and the parameter gradient of the backward pass (tcgen05 products
    with BF16 operands) vs the reference backpropagation with the same BF16 rounding points."""
    m = _mlp(langevin=False)
    rng = np.random.default_rng(2)
    Bw = 200  # not a multiple of the 128-walker GEMM tile: a ragged tail
    R0 = rng.normal(scale=1.5, size=(Bw, 17, 3))
    R1 = R0 + rng.normal(scale=0.2, size=R0.shape)
    r0, r1 = _t(R0), _t(R1)
    out = m.forward(r0)
    dout = torch.empty_like(out)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    m.nll_grad(r0, r1, out, dout, loss)
    m.zero_grad()
    m.backward(dout)
    torch.cuda.synchronize()
    want_loss, want_g, want_dout = omlp.nll_and_grad(m.params(), R0, R1, 17, 256, 2.0, 0.8, -2.0, 1.5,
                                                     acts_bf16=True)
    assert abs(loss.item() - want_loss) <= 1e-4 * abs(want_loss)
    d = dout.cpu().numpy()
    assert np.abs(d - want_dout).max() <= 1e-3 * np.abs(want_dout).max()
    g = m.grads()
    assert np.linalg.norm(g - want_g) <= 1e-3 * np.linalg.norm(want_g)
    big = np.abs(want_g) > 1e-2 * np.abs(want_g).max()
    assert (np.abs(g - want_g)[big] / np.abs(want_g)[big]).max() <= 1e-2
    m.close()


@pytest.mark.parametrize("langevin", [True, False])
def test_proposal_densities_match_oracle(langevin):
    m = _mlp(langevin=langevin)
    rng = np.random.default_rng(3)
    W = 333
    R = rng.normal(scale=1.5, size=(W, 17, 3))
    F = rng.normal(scale=2.0, size=R.shape)
    Fn = rng.normal(scale=2.0, size=R.shape)
    r, f, fn = _t(R), _t(F), _t(Fn)
    out = m.forward(r)
    rn = torch.empty_like(r)
    lqf = torch.empty(W, dtype=torch.float64, device=DEV)
    lqr = torch.empty_like(lqf)
    m.propose(r, out, 77, 5, rn, lqf, drift=f)
    out_n = m.forward(rn)
    m.reverse(r, rn, out_n, lqr, drift_new=fn)
    torch.cuda.synchronize()
    Rn, o, on = rn.cpu().numpy(), out.cpu().numpy(), out_n.cpu().numpy()
    want_f = omlp.log_q(Rn, R, o, 17, 0.8, -2.0, 1.5, F if langevin else None)
    want_r = omlp.log_q(R, Rn, on, 17, 0.8, -2.0, 1.5, Fn if langevin else None)
    np.testing.assert_allclose(lqf.cpu().numpy(), want_f, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(lqr.cpu().numpy(), want_r, rtol=1e-9, atol=1e-9)
    # the standardised noise of the drawn moves is N(0, 1)
    mu, s = omlp.head(o, 17, 0.8, -2.0, 1.5)
    sig = np.repeat(np.exp(s), 3, axis=1)
    chi = (Rn.reshape(W, -1) - R.reshape(W, -1) - mu - (sig ** 2 * F.reshape(W, -1) if langevin else 0)) / sig
    assert abs(chi.mean()) < 0.03 and abs(chi.var() - 1.0) < 0.04
    m.close()


def test_zero_network_langevin_move_is_drift_diffusion():
    """With the output layer at zero and s0 = log sqrt(tau), the learned move is
    the drift-diffusion move on the same random stream."""
    tau = 0.02
    m = _mlp(zero_head=True, s0=0.5 * math.log(tau))
    rng = np.random.default_rng(4)
    W = 129
    R = rng.normal(scale=1.5, size=(W, 17, 3))
    F = rng.normal(scale=2.0, size=R.shape)
    r, f = _t(R), _t(F)
    out = m.forward(r)
    assert float(out.abs().max()) == 0.0
    r_m, r_d = torch.empty_like(r), torch.empty_like(r)
    lq_m = torch.empty(W, dtype=torch.float64, device=DEV)
    lq_d = torch.empty_like(lq_m)
    m.propose(r, out, 31, 9, r_m, lq_m, drift=f)
    B.vmc_propose_drift(r, f, tau, 31, 9, r_d, lq_d)
    torch.cuda.synchronize()
    step = (r_d - r).abs().max().item()
    assert (r_m - r_d).abs().max().item() <= 1e-14 * max(step, 1.0)
    # log q differs only by the dropped normalisation -3N log sigma
    want = lq_d.cpu().numpy() - 3 * 17 * 0.5 * math.log(tau)
    np.testing.assert_allclose(lq_m.cpu().numpy(), want, rtol=1e-12, atol=1e-10)
    m.close()


@pytest.mark.parametrize("langevin,len2,beta", [(True, 0.0, 0.0), (True, 0.25, 0.0), (False, 0.0, 0.0),
                                               (True, 0.0, 0.3), (False, 0.0, 0.3)])
def test_esjd_gradient_matches_oracle(langevin, len2, beta):
    """Objective and dL/d(out), dL/d(out_new) of the ESJD kernel vs central
    differences of the written-out objective (oracle), on inputs where the
    acceptance is below and above 1 and with rejected (node, non-finite) moves."""
    n_elec, W = 5, 96
    m = _mlp(n_elec=n_elec, hidden=32, langevin=langevin, mm=0.7, s0=-1.5, span=1.2)
    rng = np.random.default_rng(5)
    R = rng.normal(scale=1.5, size=(W, n_elec, 3))
    F = rng.normal(scale=1.5, size=R.shape)
    Fn = rng.normal(scale=1.5, size=R.shape)
    G = Fn + rng.normal(scale=0.5, size=R.shape)  # grad log|Psi| at R'; the reverse move uses the drift Fn
    lp = rng.normal(size=W)
    lpn = lp + rng.normal(scale=2.0, size=W)
    sg = np.ones(W, np.int8)
    sg[3] = 0
    Fn[7, 2, 1] = np.nan
    G[7, 2, 1] = np.nan
    r, f, fn = _t(R), _t(F), _t(Fn)
    out = m.forward(r)
    rn = torch.empty_like(r)
    lqf = torch.empty(W, dtype=torch.float64, device=DEV)
    m.propose(r, out, 11, 3, rn, lqf, drift=f)
    out_n = m.forward(rn)
    d0, d1 = torch.empty_like(out), torch.empty_like(out)
    obj = torch.zeros(2, dtype=torch.float64, device=DEV)
    m.esjd_grad(r, rn, out, out_n, _t(lp), _t(lpn), _t(sg, torch.int8), f, fn, _t(G), d0, d1, obj,
                jump_len2=len2, speed_beta=beta)
    torch.cuda.synchronize()
    Rn, o, on = rn.cpu().numpy(), out.cpu().numpy(), out_n.cpu().numpy()
    Fn_ref = np.nan_to_num(Fn)
    sg_ref = sg.copy()
    sg_ref[7] = 0  # the kernel rejects the non-finite walker
    J, w0, w1, la = omlp.esjd_and_dout(o, on, R, Rn, lp, lpn, F, Fn_ref, sg_ref, n_elec, 0.7, -1.5, 1.2,
                                       langevin=langevin, jump_len2=len2, G_new=np.nan_to_num(G), speed_beta=beta)
    assert abs(obj[0].item() - J) <= 1e-9 * abs(J)
    A = np.where(sg_ref != 0, np.exp(np.minimum(la, 0.0)), 0.0)
    assert abs(obj[1].item() - A.mean()) <= 1e-9
    assert (la < 0).sum() > 10 and (la > 0).sum() > 10
    keep = np.abs(la) > 1e-3
    g0, g1 = d0.cpu().numpy(), d1.cpu().numpy()
    assert np.all(g0[[3, 7]] == 0) and np.all(g1[[3, 7]] == 0)
    for got, want in ((g0, w0), (g1, w1)):
        scale = np.abs(want[keep]).max()
        assert np.abs(got[keep] - want[keep]).max() <= 1e-4 * scale + 1e-12
    m.close()


def test_drift_limiter_and_acceptance_edges():
    """Limited drift against its closed form (and the small-|F| limit F), and
    acceptance of a move off |Psi| = 0."""
    rng = np.random.default_rng(8)
    W, N, tau, a = 64, 5, 0.05, 0.7
    F = rng.normal(scale=10.0, size=(W, N, 3))
    F[0] *= 1e-9
    Fb = torch.empty((W, N, 3), dtype=torch.float64, device=DEV)
    B.vmc_limit_drift(_t(F), tau, a, Fb)
    f2 = (F ** 2).sum(-1, keepdims=True)
    want = F * (-1 + np.sqrt(1 + 2 * a * tau * f2)) / (a * tau * f2)
    np.testing.assert_allclose(Fb.cpu().numpy()[1:], want[1:], rtol=1e-12)
    np.testing.assert_allclose(Fb.cpu().numpy()[0], F[0], rtol=1e-12)
    assert np.all(tau * np.linalg.norm(Fb.cpu().numpy(), axis=-1) <= np.sqrt(2 * tau / a) * (1 + 1e-12))
    B.vmc_limit_drift(_t(F), tau, 0.0, Fb)
    assert np.array_equal(Fb.cpu().numpy(), F)
    # a walker at |Psi| = 0 (log|Psi| = -inf) takes any finite proposal; a non-finite proposal is refused
    n_el = 2
    cur = {"R": _t(np.zeros((3, n_el, 3))), "log_abs_psi": _t([-np.inf, 0.0, 0.0]),
           "sign": _t([0, 1, 1], torch.int8), "grad": _t(np.zeros((3, n_el, 3))), "lap": _t(np.zeros((3, n_el))),
           "e_local": _t(np.zeros(3))}
    gn = np.ones((3, n_el, 3))
    gn[2, 1, 0] = np.nan
    new = {"R": _t(np.ones((3, n_el, 3))), "log_abs_psi": _t([-5.0, 50.0, 50.0]),
           "sign": _t([1, 1, 1], torch.int8), "grad": _t(gn), "lap": _t(np.zeros((3, n_el))),
           "e_local": _t(np.zeros(3))}
    acc = torch.empty(3, dtype=torch.int32, device=DEV)
    zero = _t(np.zeros(3))
    B.vmc_accept(1, 1, zero, zero, cur, new, accept=acc)
    assert acc.cpu().tolist() == [1, 1, 0]
    assert cur["log_abs_psi"].cpu().tolist()[:2] == [-5.0, 50.0]


def _chain_stats(r2, steps, W, dt):
    from paper_1510_00730_gb300.vmc import mean_and_error, tau_int
    t, _ = tau_int(r2)
    mean, err = mean_and_error(r2, t)
    return mean, err, t, W * steps / dt / t


def test_learned_proposal_samples_the_same_density():
    """Sampler invariance: MH with the trained proposal and plain drift-diffusion
    give the same <r^2> within 4 combined autocorrelation-corrected standard errors."""
    from paper_1510_00730_gb300.vmc import VMC, train_esjd
    wl = synth.tiny(n_walk=1024)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    tau = 0.1
    dd = VMC(ctx, wl.R, seed=21)
    dd.run(300, tau=tau, record=False)
    R_data, lp_data, F_data = dd.collect_configs(tau, 64)
    r2_d, _, _, dt_d = dd.run(2000, tau=tau)
    m = B.MLP(0, wl.n_elec, hidden=64, seed=4, mu_max=1.0, s0=0.5 * math.log(tau), s_span=2.0)
    train_esjd(m, ctx, R_data, lp_data, F_data, tau, epochs=1, batch=1024, lr=1e-4, jump_len2=0.25)
    ml = VMC(ctx, wl.R, seed=22, drift_tau=tau)
    ml.run(300, tau=tau, mlp=m, record=False)
    r2_m, _, acc, dt_m = ml.run(2000, tau=tau, mlp=m)
    md, ed, _, _ = _chain_stats(r2_d, 2000, wl.n_walk, dt_d)
    mm, em, _, _ = _chain_stats(r2_m, 2000, wl.n_walk, dt_m)
    assert acc > 0.05
    assert abs(md - mm) <= 4.0 * math.hypot(ed, em), (md, ed, mm, em)
    m.close()
    ctx.close()


# The gains of the learned move on the chlorine-like 10^5-determinant system with 8,192 walkers
# (config 5), in autocorrelation-corrected samples/s of <E_L>, over the runs of this protocol and
# of `bench.py --workload learned_proposal_100k` (1,500- and 3,000-step chains): over plain
# drift-diffusion, and over drift-diffusion with the same drift limiter. Training is not
# bit-reproducible (FP32 atomics in the weight gradients, and a training chain whose accept
# decisions follow the evaluation's rounding), so the range spans the runs' spread: nine of the
# last ten at 2.02-2.29 over plain drift-diffusion, one at 1.56.
GAIN_VS_PLAIN = (1.56, 2.58)
GAIN_VS_LIMITED = (0.68, 1.01)


def test_learned_proposal_gain_over_drift_diffusion(capsys):
    """Config 5 as the bench runs it (training on 2^20 configurations of the plain
    chain, then 1,500-step chains from the same walkers): the learned move's gains over
    plain and over limited drift-diffusion lie within the range of the reported runs,
    widened by three of this run's autocorrelation-corrected standard errors (Sokal's
    error of tau_int, averaged over the walkers)."""
    from paper_1510_00730_gb300.vmc import learned_vs_drift_diffusion
    wl = synth.chlorine_like_100k(n_walk=8192)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    r = learned_vs_drift_diffusion(ctx, wl.R, 3e-5, 1500, warmup=100)
    ctx.close()
    g, eg = r["gain"], r["gain_err"]
    gl, egl = r["gain_vs_limited"], r["gain_vs_limited_err"]
    with capsys.disabled():
        print("\nlearned proposal, chlorine-like 1e5: gain %.2f +- %.2f over plain drift-diffusion, %.2f +- %.2f "
              "over the limited one; tau_int(E_L) %.0f / %.0f / %.0f; acceptance %.2f / %.2f / %.2f"
              % (g, eg, gl, egl, r["learned"]["tau_int"], r["drift_diffusion"]["tau_int"],
                 r["drift_diffusion_limited"]["tau_int"], r["learned"]["acceptance"],
                 r["drift_diffusion"]["acceptance"], r["drift_diffusion_limited"]["acceptance"]))
    assert GAIN_VS_PLAIN[0] - 3 * eg <= g <= GAIN_VS_PLAIN[1] + 3 * eg, (g, eg)
    assert GAIN_VS_LIMITED[0] - 3 * egl <= gl <= GAIN_VS_LIMITED[1] + 3 * egl, (gl, egl)
    assert r["learned"]["acceptance"] > 0.05


def test_learned_proposal_chain_on_a_small_system(capsys):
    """The whole learned-move loop on the 4-electron system: a drift-diffusion chain,
    training, and both chains from the same walkers; the learned chain accepts moves and
    both samples/s estimates are finite."""
    from paper_1510_00730_gb300.vmc import VMC, measure_chain, train_esjd
    wl = synth.tiny(n_walk=2048)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_MIXED)
    tau = 0.1
    dd = VMC(ctx, wl.R, seed=31, drift_tau=tau)
    dd.run(400, tau=tau, record=False)
    R_eq = dd.cur["R"].clone()
    R_data, lp_data, F_data = dd.collect_configs(tau, 128)
    m = B.MLP(0, wl.n_elec, hidden=256, seed=3, mu_max=1.0, s0=0.5 * math.log(tau), s_span=3.0)
    train_esjd(m, ctx, R_data, lp_data, F_data, tau, epochs=3, batch=2048, lr=3e-4, speed_beta=0.1,
               target_acc=0.4)
    base = measure_chain(ctx, R_eq, 1500, tau, seed=5)
    learned = measure_chain(ctx, R_eq, 1500, tau, mlp=m, seed=6)
    gain = learned["samples_per_s"] / base["samples_per_s"]
    with capsys.disabled():
        print("\nlearned proposal on %s: acceptance %.3f vs %.3f, tau_int(E_L) %.1f vs %.1f, "
              "%.3f vs %.3f ms/step, gain %.2f" % (wl.name, learned["acceptance"], base["acceptance"],
                                                  learned["tau_int"], base["tau_int"], learned["ms_per_step"],
                                                  base["ms_per_step"], gain))
    assert learned["acceptance"] > 0.05 and np.isfinite(gain) and gain > 0
    m.close()
    ctx.close()


def test_chain_resumes_from_checkpoint(tmp_path):
    """A chain resumed from its checkpoint continues the uninterrupted chain: the
    same counter-based random numbers and the same network, so the positions
    after further learned and drift-diffusion steps agree to rounding."""
    from paper_1510_00730_gb300.vmc import VMC, resume_checkpoint, save_checkpoint
    wl = synth.tiny(n_walk=256)
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    tau = 0.1
    m = B.MLP(0, wl.n_elec, hidden=32, seed=4, mu_max=1.0, s0=0.5 * math.log(tau), s_span=2.0, zero_head=False)
    a = VMC(ctx, wl.R, seed=41, drift_tau=tau)
    a.run(20, tau=tau, mlp=m, mix_drift=0.3, record=False)
    p = tmp_path / "chain.bin"
    save_checkpoint(p, a, m)
    m2 = B.MLP(0, wl.n_elec, hidden=32, seed=99, mu_max=1.0, s0=0.5 * math.log(tau), s_span=2.0)
    b = resume_checkpoint(p, ctx, m2)
    assert b.step_count == a.step_count and np.array_equal(m2.params(), m.params())
    for k in range(10):
        if k % 3 == 2:
            a.step_drift(tau)
            b.step_drift(tau)
        else:
            a.step_mlp(m)
            b.step_mlp(m2)
    torch.cuda.synchronize()
    ra, rb = a.cur["R"].cpu().numpy(), b.cur["R"].cpu().numpy()
    same = np.abs(ra - rb).max(axis=(1, 2)) <= 1e-10
    assert same.mean() >= 0.99, same.mean()  # an acceptance test within rounding of its threshold may flip
    m.close()
    m2.close()
    ctx.close()
