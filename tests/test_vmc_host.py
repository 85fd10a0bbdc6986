"""Host-side pieces of the VMC driver and learned proposal: the counter-based
generator against its published known answers (and an independent
implementation), the reference perceptron's gradient against finite
differences, and the autocorrelation-time estimator against a closed form."""
from __future__ import annotations

import numpy as np

from oracle import mlp as omlp
from paper_1510_00730_gb300 import binding
from paper_1510_00730_gb300.vmc import tau_int

M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85


def philox_py(ctr, key):
    """Philox4x32-10 written from its definition (Salmon et al., SC'11)."""
    c, k = list(ctr), list(key)
    for _ in range(10):
        p0, p1 = M0 * c[0], M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & 0xFFFFFFFF, p1 & 0xFFFFFFFF, ((p0 >> 32) ^ c[3] ^ k[1]) & 0xFFFFFFFF,
             p0 & 0xFFFFFFFF]
        k = [(k[0] + W0) & 0xFFFFFFFF, (k[1] + W1) & 0xFFFFFFFF]
    return c


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Random123 distribution)."""
    kat = [([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
           ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
           ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
            [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1])]
    for ctr, key, want in kat:
        assert philox_py(ctr, key) == want
        assert binding.philox4x32_10(ctr, key) == want
    rng = np.random.default_rng(0)
    for _ in range(50):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, 4)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, 2)]
        assert binding.philox4x32_10(ctr, key) == philox_py(ctr, key)


def test_reference_mlp_gradient_vs_finite_differences():
    n_elec, H = 3, 8
    rng = np.random.default_rng(1)
    n_par = 9 * H + H + H * H + H + H * 12 + 12
    p = rng.normal(scale=0.3, size=n_par)
    R0 = rng.normal(size=(5, n_elec, 3))
    R1 = R0 + rng.normal(scale=0.3, size=R0.shape)
    args = (R0, R1, n_elec, H, 2.0, 0.8, -1.0, 1.5)
    loss, g, _ = omlp.nll_and_grad(p, *args, weights_bf16=False)
    for i in rng.choice(n_par, 40, replace=False):
        e = np.zeros(n_par); e[i] = 1e-6
        fd = (omlp.nll_and_grad(p + e, *args, weights_bf16=False)[0] -
              omlp.nll_and_grad(p - e, *args, weights_bf16=False)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def _one_unit_net():
    """n_elec = 1 (3 inputs, 4 outputs), one hidden unit per layer: W1 = e_0, W2 = 1,
    W3 = e_0, zero biases, so out[0] = tanh(tanh(x_0)) along a single path."""
    W1 = [1.0, 0.0, 0.0]
    W3 = [1.0, 0.0, 0.0, 0.0]
    return np.array(W1 + [0.0] + [1.0] + [0.0] + W3 + [0.0] * 4)


def test_bf16_activation_rounding_points():
    """The tensor-core arithmetic (acts_bf16): each product's activation operand is
    rounded to BF16, 8 significant bits, nearest even. Hand-worked on x_0 = 1 + 2^-10:
    - x_0 rounds to 1.0, so h1 = tanh(1) = 0.76159415595..., 194.968 units of 2^-8;
    - h1 rounds to 195 * 2^-8 = 0.76171875, so h2 = tanh(0.76171875) = 0.64208822...,
      164.375 units of 2^-8;
    - h2 rounds to 164 * 2^-8 = 0.640625, which is the output exactly.
    Without the rounding the output is tanh(tanh(1 + 2^-10))."""
    p = _one_unit_net()
    R = np.array([[[1.0 + 2.0 ** -10, 0.0, 0.0]]])
    out, (x, h1, h2, *_) = omlp.forward(p, R, 1, 1, 1.0, weights_bf16=True, acts_bf16=True)
    assert out[0, 0] == 0.640625 and np.all(out[0, 1:] == 0.0)
    assert h1[0, 0] == np.tanh(1.0)  # x rounded before the first product
    assert h2[0, 0] == np.tanh(0.76171875)  # h1 rounded before the second
    plain, _ = omlp.forward(p, R, 1, 1, 1.0, weights_bf16=True, acts_bf16=False)
    assert plain[0, 0] == np.tanh(np.tanh(1.0 + 2.0 ** -10))


def test_bf16_activation_gradient_stays_near_the_exact_one():
    """Rounding every product's operands to BF16 moves the backpropagated gradient by a
    few 2^-9 relative rounding errors, never by more than a percent of its norm."""
    rng = np.random.default_rng(4)
    n_e, H = 3, 16
    n_in, n_out = 3 * n_e, 4 * n_e
    p = rng.normal(scale=0.4, size=n_in * H + H + H * H + H + H * n_out + n_out)
    R0 = rng.normal(scale=1.2, size=(64, n_e, 3))
    R1 = R0 + rng.normal(scale=0.2, size=R0.shape)
    args = (R0, R1, n_e, H, 2.0, 0.8, -2.0, 1.5)
    l0, g0, _ = omlp.nll_and_grad(p, *args)
    l1, g1, _ = omlp.nll_and_grad(p, *args, acts_bf16=True)
    assert abs(l1 - l0) <= 1e-2 * abs(l0)
    assert 0.0 < np.linalg.norm(g1 - g0) <= 1e-2 * np.linalg.norm(g0)


def test_tau_int_ar1_closed_form():
    """For an AR(1) series x_t = phi x_{t-1} + noise, tau_int = (1 + phi) / (1 - phi)."""
    rng = np.random.default_rng(2)
    for phi in (0.0, 0.5, 0.8):
        T, W = 4000, 64
        x = np.zeros((T, W))
        e = rng.normal(size=(T, W))
        for t in range(1, T):
            x[t] = phi * x[t - 1] + e[t]
        tau, _ = tau_int(x[200:])
        want = (1 + phi) / (1 - phi)
        assert abs(tau - want) < 0.12 * want, (phi, tau, want)


def test_log_q_is_the_gaussian_density():
    """log_q plus the normalisation equals the library's multivariate normal log-density."""
    from scipy.stats import multivariate_normal
    rng = np.random.default_rng(3)
    n_elec, B = 3, 4
    out = rng.normal(scale=0.7, size=(B, 4 * n_elec))
    R = rng.normal(size=(B, n_elec, 3))
    F = rng.normal(size=(B, n_elec, 3))
    Rt = R + rng.normal(scale=0.3, size=R.shape)
    mm, s0, span = 0.8, -1.2, 1.5
    for drift in (None, F):
        lq = omlp.log_q(Rt, R, out, n_elec, mm, s0, span, drift)
        for w in range(B):
            s = s0 + span * np.tanh(out[w, 3 * n_elec:])
            sig = np.repeat(np.exp(s), 3)
            mean = R[w].ravel() + sig * mm * np.tanh(out[w, :3 * n_elec])
            if drift is not None:
                mean = mean + sig ** 2 * F[w].ravel()
            want = multivariate_normal(mean=mean, cov=np.diag(sig ** 2)).logpdf(Rt[w].ravel())
            assert abs(lq[w] - 1.5 * n_elec * np.log(2 * np.pi) - want) < 1e-10 * max(1.0, abs(want))


def _esjd_case(rng, B=6, n_elec=3, langevin=True, zero_out=False):
    out = np.zeros((B, 4 * n_elec)) if zero_out else rng.normal(scale=0.5, size=(B, 4 * n_elec))
    out_new = np.zeros_like(out) if zero_out else rng.normal(scale=0.5, size=out.shape)
    R = rng.normal(size=(B, n_elec, 3))
    F = rng.normal(size=R.shape)
    Rn = R + rng.normal(scale=0.2, size=R.shape)
    Fn = rng.normal(size=R.shape)
    lp = rng.normal(size=B)
    lpn = lp + rng.normal(scale=0.5, size=B)
    return out, out_new, R, Rn, lp, lpn, F, Fn, np.ones(B, np.int8)


def test_esjd_log_alpha_reduces_to_drift_diffusion():
    """With zero outputs and s0 = log sqrt(tau), the Langevin-form move is the
    drift-diffusion move, and log alpha is its Metropolis-Hastings ratio."""
    rng = np.random.default_rng(4)
    tau = 0.03
    out, out_new, R, Rn, lp, lpn, F, Fn, sg = _esjd_case(rng, zero_out=True)
    _, _, _, la = omlp.esjd_and_dout(out, out_new, R, Rn, lp, lpn, F, Fn, sg, 3, 1.0, 0.5 * np.log(tau), 2.0)
    fwd = ((Rn - R - tau * F) ** 2).sum((1, 2)) / (2 * tau)
    rev = ((R - Rn - tau * Fn) ** 2).sum((1, 2)) / (2 * tau)
    np.testing.assert_allclose(la, 2 * (lpn - lp) - rev + fwd, rtol=1e-12, atol=1e-12)


def test_esjd_symmetric_move_log_alpha():
    """Without the Langevin term and with equal scales at both ends, the
    proposal is symmetric and log alpha = 2 (log|Psi'| - log|Psi|)."""
    rng = np.random.default_rng(5)
    out, out_new, R, Rn, lp, lpn, F, Fn, sg = _esjd_case(rng, langevin=False, zero_out=True)
    _, _, _, la = omlp.esjd_and_dout(out, out_new, R, Rn, lp, lpn, F, Fn, sg, 3, 1.0, -1.0, 2.0, langevin=False)
    np.testing.assert_allclose(la, 2 * (lpn - lp), rtol=1e-12, atol=1e-12)


def test_esjd_gradient_closed_form_when_always_accepted():
    """When every move is accepted (A = 1) and |Psi| is flat at R', J = mean |R' - R|^2
    with R' - R = mu + sigma chi, so dJ/dmu_c = 2 dR_c and dJ/ds_e = 2 |dR_e|^2."""
    rng = np.random.default_rng(6)
    n_elec, B, mm, s0, span = 3, 6, 0.7, -1.0, 2.0
    out, out_new, R, Rn, lp, lpn, F, Fn, sg = _esjd_case(rng, B=B, n_elec=n_elec)
    lp[:] = -200.0
    lpn[:] = 0.0
    Fn[:] = 0.0
    J, d0, d1, la = omlp.esjd_and_dout(out, out_new, R, Rn, lp, lpn, F, Fn, sg, n_elec, mm, s0, span,
                                       langevin=False)
    assert (la > 0).all()
    dR = (Rn - R).reshape(B, -1)
    tm, ts = np.tanh(out[:, :3 * n_elec]), np.tanh(out[:, 3 * n_elec:])
    sig = np.exp(s0 + span * ts)
    want_mu = -2 * dR * np.repeat(sig, 3, axis=1) * mm * (1 - tm ** 2) / B
    want_s = -2 * (dR.reshape(B, n_elec, 3) ** 2).sum(-1) * span * (1 - ts ** 2) / B
    np.testing.assert_allclose(d0[:, :3 * n_elec], want_mu, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(d0[:, 3 * n_elec:], want_s, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(d1, 0.0, atol=1e-9)
    assert abs(J - (dR ** 2).sum(1).mean()) < 1e-12 * J


def test_speed_measure_gradient_closed_form_when_always_accepted():
    """With every move accepted, the speed measure is beta * 3 sum_e s_e, whose
    gradient is 3 beta on each log-scale and zero elsewhere."""
    rng = np.random.default_rng(7)
    n_elec, B, mm, s0, span, beta = 3, 6, 0.7, -1.0, 2.0, 0.4
    out, out_new, R, Rn, lp, lpn, F, Fn, sg = _esjd_case(rng, B=B, n_elec=n_elec)
    lp[:] = -200.0
    lpn[:] = 0.0
    Fn[:] = 0.0
    J, d0, d1, la = omlp.esjd_and_dout(out, out_new, R, Rn, lp, lpn, F, Fn, sg, n_elec, mm, s0, span,
                                       langevin=False, speed_beta=beta)
    assert (la > 0).all()
    ts = np.tanh(out[:, 3 * n_elec:])
    np.testing.assert_allclose(d0[:, :3 * n_elec], 0.0, atol=1e-9)
    np.testing.assert_allclose(d0[:, 3 * n_elec:], -3 * beta * span * (1 - ts ** 2) / B, rtol=1e-6)
    np.testing.assert_allclose(d1, 0.0, atol=1e-9)
    assert abs(J - beta * 3 * (s0 + span * ts).sum(1).mean()) < 1e-12


def test_checkpoint_round_trip(tmp_path):
    """The flat chain checkpoint reads back exactly; a wrong magic or a truncated file is refused."""
    import pytest
    import torch
    from types import SimpleNamespace

    from paper_1510_00730_gb300.vmc import read_checkpoint, save_checkpoint
    rng = np.random.default_rng(9)
    R = rng.normal(size=(5, 3, 3))
    vmc = SimpleNamespace(W=5, N=3, seed=123456789012, step_count=77, drift_a=1.0, drift_tau=3e-5,
                          cur={"R": torch.from_numpy(R)})
    params = rng.normal(size=41).astype(np.float32)
    mlp = SimpleNamespace(params=lambda: params)
    p = tmp_path / "chain.bin"
    save_checkpoint(p, vmc, mlp)
    ck = read_checkpoint(p)
    assert (ck["W"], ck["N"], ck["seed"], ck["step"], ck["drift_a"], ck["drift_tau"]) == (5, 3, 123456789012, 77,
                                                                                        1.0, 3e-5)
    assert np.array_equal(ck["R"], R) and np.array_equal(ck["params"], params)
    vmc.drift_tau = None
    save_checkpoint(p, vmc)
    ck = read_checkpoint(p)
    assert ck["drift_tau"] is None and ck["params"].size == 0
    data = p.read_bytes()
    (tmp_path / "short.bin").write_bytes(data[:-8])
    with pytest.raises(ValueError):
        read_checkpoint(tmp_path / "short.bin")
    (tmp_path / "bad.bin").write_bytes(b"NOTACKPT" + data[8:])
    with pytest.raises(ValueError):
        read_checkpoint(tmp_path / "bad.bin")
