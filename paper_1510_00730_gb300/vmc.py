"""Variational Monte Carlo around the hot path, with a learned proposal.

One Monte Carlo step moves all electrons of every walker (the unit the paper
times in Sec. 4: Psi, the drift and E_L at every step). The loop below runs on
the host; every numeric step runs in libmdet.so's kernels: the proposal and its
densities (mdet_vmc_*), the wavefunction, drift and local energy
(mdet_evaluate), the Metropolis-Hastings acceptance, and the perceptron's
forward, backward and Adam kernels (mdet_mlp_*).

Because every move is accepted with the exact |Psi(R')/Psi(R)|^2 and both
proposal densities, the chain samples |Psi|^2 whichever proposal is used; the
learned proposal can only change how fast the chain decorrelates.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import binding as B


class VMC:
    """Walkers of one context, with current and proposed state on the device."""

    def __init__(self, ctx, R0, seed=12345, drift_a=1.0, drift_tau=None):
        """drift_a: Umrigar-Nightingale-Runge drift limiting (0 = off) applied
        to the drift of both kinds of moves; the limiting time step is the
        drift-diffusion tau (drift_tau for the learned moves when no
        drift-diffusion step has set it)."""
        import torch
        self.torch = torch
        self.ctx = ctx
        self.dev = torch.device("cuda", ctx.device)
        R0 = torch.as_tensor(np.ascontiguousarray(R0), dtype=torch.float64, device=self.dev) \
            if not isinstance(R0, torch.Tensor) else R0.contiguous()
        self.W, self.N = R0.shape[0], R0.shape[1]
        self.seed = int(seed)
        self.step_count = 0
        self.cur = ctx.alloc_outputs(self.W)
        self.cur["R"] = R0.clone()
        self.new = ctx.alloc_outputs(self.W)
        self.new["R"] = torch.empty_like(R0)
        ctx.evaluate(self.cur["R"], out=self.cur)
        self.lqf = torch.empty(self.W, dtype=torch.float64, device=self.dev)
        self.lqr = torch.empty_like(self.lqf)
        self.acc = torch.empty(self.W, dtype=torch.int32, device=self.dev)
        self.nacc = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.r2 = torch.empty(self.W, dtype=torch.float64, device=self.dev)
        self.out0 = self.out1 = None
        self.out_owner = None
        self.drift_a = float(drift_a)
        self.drift_tau = drift_tau
        self.fb0 = torch.empty_like(R0)
        self.fb1 = torch.empty_like(R0)

    # ---- one all-electron step of each kind -------------------------------
    def _limit(self, F, out, tau):
        B.vmc_limit_drift(F, tau, self.drift_a, out)
        return out

    def step_drift(self, tau):
        self.out_owner = None  # positions may change: the cached network output is stale
        if self.drift_tau is None:
            self.drift_tau = tau
        c, n = self.cur, self.new
        B.vmc_propose_drift(c["R"], self._limit(c["grad"], self.fb0, tau), tau, self.seed, self.step_count, n["R"],
                            self.lqf)
        self.ctx.evaluate(n["R"], out=n)
        B.vmc_reverse_drift(c["R"], n["R"], self._limit(n["grad"], self.fb1, tau), tau, self.lqr)
        B.vmc_accept(self.seed, self.step_count, self.lqf, self.lqr, c, n, accept=self.acc, n_accept=self.nacc)
        self.step_count += 1

    def step_mlp(self, mlp):
        """One learned move. The network output at the current positions is
        kept across steps (rows of accepted walkers are taken from the output
        at the proposed positions), so a step runs one forward pass."""
        c, n = self.cur, self.new
        if self.out0 is None or self.out_owner is not mlp:
            self.out0 = mlp.forward(c["R"], out=self.out0)
            self.out_owner = mlp
        t = self.drift_tau
        if t is None:
            raise ValueError("learned moves need drift_tau (the limiting time step of the drift)")
        mlp.propose(c["R"], self.out0, self.seed, self.step_count, n["R"], self.lqf,
                    drift=self._limit(c["grad"], self.fb0, t))
        self.ctx.evaluate(n["R"], out=n)
        self.out1 = mlp.forward(n["R"], out=self.out1)
        mlp.reverse(c["R"], n["R"], self.out1, self.lqr, drift_new=self._limit(n["grad"], self.fb1, t))
        B.vmc_accept(self.seed, self.step_count, self.lqf, self.lqr, c, n, accept=self.acc, n_accept=self.nacc)
        B.vmc_select_rows(self.acc, self.out1, self.out0)
        self.step_count += 1

    # ---- chains ------------------------------------------------------------
    def run(self, n_steps, tau=None, mlp=None, mix_drift=0.0, record=True, rng=None):
        """n_steps steps; with mlp, a fraction mix_drift of the steps (chosen
        independently of the state) are drift-diffusion steps with tau. Returns
        the recorded observables [n_steps][W] (r^2, E_L), the acceptance rate
        and the wall time of the steps (device-synchronised)."""
        torch = self.torch
        rng = rng or np.random.default_rng(self.seed + 17)
        r2 = torch.empty((n_steps, self.W), dtype=torch.float64, device=self.dev) if record else None
        el = torch.empty_like(r2) if record else None
        self.nacc.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(n_steps):
            if mlp is not None and not (mix_drift > 0.0 and rng.random() < mix_drift):
                self.step_mlp(mlp)
            else:
                self.step_drift(tau)
            if record:
                B.vmc_r2(self.cur["R"], r2[s])
                el[s].copy_(self.cur["e_local"])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        acc = int(self.nacc.item()) / float(n_steps * self.W)
        if not record:
            return None, None, acc, dt
        return r2.cpu().numpy(), el.cpu().numpy(), acc, dt

    def collect_configs(self, tau, n_steps, every=1):
        """Configurations of the drift-diffusion chain with their log|Psi| and
        drift, one per walker every `every` steps: [M][N][3], [M], [M][N][3]
        (device, M = W * (n_steps // every))."""
        torch = self.torch
        Rs, lps, Fs = [], [], []
        for s in range(n_steps):
            self.step_drift(tau)
            if (s + 1) % every == 0:
                Rs.append(self.cur["R"].clone())
                lps.append(self.cur["log_abs_psi"].clone())
                Fs.append(self.cur["grad"].clone())
        return torch.cat(Rs), torch.cat(lps), torch.cat(Fs)

    def collect_pairs(self, tau, n_steps, lag):
        """Configurations of the drift-diffusion chain paired at the given lag:
        (R_t, R_{t+lag}) for every walker, as two [pairs][N][3] device tensors."""
        torch = self.torch
        ring = [self.cur["R"].clone() for _ in range(lag)]
        R0, R1 = [], []
        for s in range(n_steps + lag):
            self.step_drift(tau)
            if s >= lag:
                R0.append(ring[s % lag].clone())
                R1.append(self.cur["R"].clone())
            ring[s % lag].copy_(self.cur["R"])
        return torch.cat(R0), torch.cat(R1)


_CKPT_MAGIC = b"MDETVMC1"


def save_checkpoint(path, vmc, mlp=None):
    """Write the chain state as one flat little-endian binary: the magic
    MDETVMC1, then int64 walkers, electrons, seed, step, parameter count
    (0 without a network), float64 drift_a, drift_tau (NaN when unset), the
    positions [W][N][3] float64 and the network's FP32 master parameters. The
    random numbers are counter-based (Philox keyed by seed and step), so seed
    and step are the whole generator state."""
    import struct
    R = vmc.cur["R"].detach().cpu().numpy().astype("<f8")
    params = mlp.params().astype("<f4") if mlp is not None else np.zeros(0, "<f4")
    tau = float("nan") if vmc.drift_tau is None else float(vmc.drift_tau)
    with open(path, "wb") as f:
        f.write(_CKPT_MAGIC)
        f.write(struct.pack("<5q2d", vmc.W, vmc.N, vmc.seed, vmc.step_count, params.size, vmc.drift_a, tau))
        f.write(R.tobytes())
        f.write(params.tobytes())


def read_checkpoint(path):
    """The fields written by save_checkpoint, as a dict (host arrays)."""
    import struct
    with open(path, "rb") as f:
        if f.read(8) != _CKPT_MAGIC:
            raise ValueError("not a chain checkpoint: " + str(path))
        W, N, seed, step, n_par, drift_a, tau = struct.unpack("<5q2d", f.read(56))
        R = np.frombuffer(f.read(W * N * 3 * 8), dtype="<f8").reshape(W, N, 3).copy()
        params = np.frombuffer(f.read(n_par * 4), dtype="<f4").copy()
        if R.size != W * N * 3 or params.size != n_par:
            raise ValueError("truncated chain checkpoint: " + str(path))
    return dict(W=W, N=N, seed=seed, step=step, R=R, params=params, drift_a=drift_a,
                drift_tau=None if tau != tau else tau)


def resume_checkpoint(path, ctx, mlp=None):
    """A VMC chain on ctx continuing from the checkpoint: positions, seed, step
    and drift settings restored, the wavefunction re-evaluated at the positions,
    and the network's parameters loaded into mlp when given."""
    ck = read_checkpoint(path)
    if ck["N"] != ctx.n_up + ctx.n_dn:
        raise ValueError("checkpoint has %d electrons, the context %d" % (ck["N"], ctx.n_up + ctx.n_dn))
    v = VMC(ctx, ck["R"], seed=ck["seed"], drift_a=ck["drift_a"], drift_tau=ck["drift_tau"])
    v.step_count = ck["step"]
    if mlp is not None:
        if ck["params"].size != mlp.n_params:
            raise ValueError("checkpoint network has %d parameters, the given one %d" % (ck["params"].size,
                                                                                       mlp.n_params))
        mlp.set_params(ck["params"])
    return v


def train_proposal(mlp, R0, R1, epochs=4, batch=8192, lr=1e-3, seed=0, log=None):
    """Maximum-likelihood fit of the perceptron's Gaussian move to observed
    moves R0 -> R1 (Adam on minibatches; the loss is the mean negative
    log-likelihood). Returns the loss history per epoch."""
    import torch
    dev = R0.device
    n = R0.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    out = torch.empty(batch, 4 * mlp.n_elec, dtype=torch.float32, device=dev)
    dout = torch.empty_like(out)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    hist = []
    t = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        tot, cnt = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            r0, r1 = R0.index_select(0, idx).contiguous(), R1.index_select(0, idx).contiguous()
            mlp.forward(r0, out=out)
            mlp.nll_grad(r0, r1, out, dout, loss)
            mlp.zero_grad()
            mlp.backward(dout)
            t += 1
            mlp.adam(lr, t)
            tot += float(loss.item())
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log("epoch %d: nll %.4f" % (ep, hist[-1]))
    return hist


def train_esjd(mlp, ctx, R_data, lp_data, F_data, drift_tau, epochs=2, batch=8192, lr=1e-4, jump_len2=0.0,
               drift_a=1.0, speed_beta=0.0, target_acc=None, beta_rate=0.05, seed=0, log=None):
    """Train the proposal to maximise the acceptance-weighted squared jump
    distance E[A |R' - R|^2] over configurations of the plain chain (R_data,
    with their log|Psi| and drift in lp_data, F_data): per minibatch one proposal, one
    evaluation of Psi and its drift at the proposed points (the hot path),
    the reparametrisation gradient (mdet_mlp_esjd_grad), backward passes at
    both points and an Adam step. jump_len2 > 0 weights each electron's
    squared jump by 1 / (|R_e|^2 + jump_len2). speed_beta > 0 trains on the
    generalised speed measure instead (mdet_mlp_esjd_grad); with target_acc the
    weight beta of its entropy term follows the minibatch acceptance,
    beta <- beta exp(beta_rate (acceptance - target_acc)). The moves use the
    drift limited with (drift_tau, drift_a), as the chain does. Returns the
    objective and the mean acceptance per epoch."""
    import torch
    dev = R_data.device
    n = R_data.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    N = mlp.n_elec
    out0 = torch.empty(batch, 4 * N, dtype=torch.float32, device=dev)
    out1, d0, d1 = torch.empty_like(out0), torch.empty_like(out0), torch.empty_like(out0)
    r1 = torch.empty(batch, N, 3, dtype=torch.float64, device=dev)
    f0, f1 = torch.empty_like(r1), torch.empty_like(r1)
    lqf = torch.empty(batch, dtype=torch.float64, device=dev)
    ev = ctx.alloc_outputs(batch)
    obj = torch.zeros(2, dtype=torch.float64, device=dev)
    hist, t = [], 0
    beta = float(speed_beta)
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        tot, tacc, cnt = 0.0, 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            r0, lp0 = R_data.index_select(0, idx).contiguous(), lp_data.index_select(0, idx).contiguous()
            B.vmc_limit_drift(F_data.index_select(0, idx), drift_tau, drift_a, f0)
            t += 1
            mlp.forward(r0, out=out0)
            mlp.propose(r0, out0, seed + 7919, t, r1, lqf, drift=f0)
            ctx.evaluate(r1, out=ev)
            B.vmc_limit_drift(ev["grad"], drift_tau, drift_a, f1)
            mlp.forward(r1, out=out1)
            mlp.esjd_grad(r0, r1, out0, out1, lp0, ev["log_abs_psi"], ev["sign"], f0, f1, ev["grad"], d0, d1, obj,
                          jump_len2=jump_len2, speed_beta=beta)
            mlp.zero_grad()
            mlp.backward(d1)
            mlp.forward(r0, out=out0)
            mlp.backward(d0)
            mlp.adam(lr, t)
            j, acc = obj.tolist()
            tot += j
            tacc += acc
            cnt += 1
            if beta > 0 and target_acc is not None:
                beta *= math.exp(beta_rate * (acc - target_acc))
        hist.append((tot / max(cnt, 1), tacc / max(cnt, 1)))
        if log:
            log("epoch %d: objective %.5f acceptance %.3f beta %.4g" % (ep, hist[-1][0], hist[-1][1], beta))
    return hist


def measure_chain(ctx, R0, n_steps, tau, mlp=None, mix_drift=0.0, seed=11, warmup=100, drift_a=1.0):
    """Run a chain from R0 (warmup steps, then n_steps recorded) and return its
    acceptance, Sokal's tau_int of E_L, the step time (a separate run of up to
    200 unrecorded steps) and the autocorrelation-corrected samples/s of <E_L>
    = walkers / (seconds per step * tau_int), with <r^2> and its error."""
    import torch
    v = VMC(ctx, R0.clone(), seed=seed, drift_a=drift_a, drift_tau=tau)
    v.run(warmup, tau=tau, mlp=mlp, mix_drift=mix_drift, record=False)
    r2, el, acc, _ = v.run(n_steps, tau=tau, mlp=mlp, mix_drift=mix_drift)
    k = min(n_steps, 200)
    _, _, _, dt = v.run(k, tau=tau, mlp=mlp, mix_drift=mix_drift, record=False)
    t_el, win = tau_int(el)
    t_r2, _ = tau_int(r2)
    m, e = mean_and_error(r2, t_r2)
    sps = dt / k
    t_err = tau_int_error(t_el, win, *np.asarray(el).shape)
    sp = v.W / sps / t_el
    return {"acceptance": acc, "tau_int": t_el, "tau_int_err": t_err, "tau_window": win, "tau_int_r2": t_r2,
            "ms_per_step": 1e3 * sps, "samples_per_s": sp, "samples_per_s_err": sp * t_err / t_el,
            "r2": m, "r2_err": e, "steps": n_steps}


def tau_int_error(tau, M, n_steps, n_walkers):
    """Statistical error of tau_int from Sokal's window estimate, var(tau) ~ 2 (2M + 1) / N tau^2
    for one series of N steps (Madras and Sokal, J. Stat. Phys. 50, 109 (1988)); the
    autocorrelation here is averaged over independent walkers, which divides the variance
    by their number."""
    return float(tau * np.sqrt(2.0 * (2 * M + 1) / (n_steps * max(n_walkers, 1))))


def learned_vs_drift_diffusion(ctx, R, tau, n_chain, warmup=100, n_configs=1 << 20, hidden=256, seed=3):
    """The learned proposal against drift-diffusion on one context (config 5 of the brief,
    run by `bench.py --workload learned_proposal_100k` and by the GPU tests):
    1. 500 steps of drift-diffusion with the drift limiter equilibrate the walkers R;
    2. the same chain collects about n_configs configurations;
    3. the perceptron is trained on them on the GPU (generalised speed measure, target
       acceptance 0.5, 3 epochs);
    4. three chains of n_chain recorded steps run from the same equilibrated walkers:
       plain drift-diffusion (no drift capping), drift-diffusion with the limiter, and the
       learned move with the limiter.
    Returns the three chains' measurements, the gains of the learned move in
    autocorrelation-corrected samples/s of <E_L> with their errors (relative errors of the
    two samples/s added in quadrature), and the training record."""
    import torch
    W = len(R)
    dd = VMC(ctx, R, seed=2, drift_tau=tau)
    dd.run(500, tau=tau, record=False)
    R_eq = dd.cur["R"].clone()
    t0 = time.perf_counter()
    R_data, lp_data, F_data = dd.collect_configs(tau, max(1, n_configs // W))
    torch.cuda.synchronize()
    collect_s = time.perf_counter() - t0
    mlp = B.MLP(ctx.device, ctx.n_up + ctx.n_dn, hidden=hidden, seed=seed, mu_max=1.0, s0=0.5 * math.log(tau), s_span=3.0)
    try:
        t0 = time.perf_counter()
        hist = train_esjd(mlp, ctx, R_data, lp_data, F_data, tau, epochs=3, batch=min(W, 8192), lr=1e-4,
                          speed_beta=0.1, target_acc=0.5)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        base = measure_chain(ctx, R_eq, n_chain, tau, seed=5, warmup=warmup, drift_a=0.0)
        limited = measure_chain(ctx, R_eq, n_chain, tau, seed=5, warmup=warmup, drift_a=1.0)
        learned = measure_chain(ctx, R_eq, n_chain, tau, mlp=mlp, seed=6, warmup=warmup, drift_a=1.0)
    finally:
        mlp.close()

    def gain(a, b):
        g = a["samples_per_s"] / b["samples_per_s"]
        r = math.hypot(a["samples_per_s_err"] / a["samples_per_s"], b["samples_per_s_err"] / b["samples_per_s"])
        return g, g * r

    g_plain, e_plain = gain(learned, base)
    g_lim, e_lim = gain(learned, limited)
    return {"learned": learned, "drift_diffusion": base, "drift_diffusion_limited": limited,
            "gain": g_plain, "gain_err": e_plain, "gain_vs_limited": g_lim, "gain_vs_limited_err": e_lim,
            "training_configs": int(R_data.shape[0]), "collect_s": collect_s, "train_s": train_s,
            "objective_acceptance_per_epoch": hist}


def tau_int(x, c=5.0):
    """Integrated autocorrelation time of per-walker series x[step][walker]
    with Sokal's automatic window: the smallest M with M >= c tau(M), where
    tau(M) = 1 + 2 sum_{t=1..M} rho(t) and rho is the autocorrelation averaged
    over walkers. The series are centred on the mean over all walkers and
    steps (the walkers sample one stationary distribution): centring each
    walker on its own mean would hide the correlation of a chain that seldom
    moves. Returns (tau, M)."""
    x = np.asarray(x, dtype=np.float64)
    T = x.shape[0]
    y = x - x.mean()
    n = 1 << int(np.ceil(np.log2(2 * T)))
    f = np.fft.rfft(y, n=n, axis=0)
    acf = np.fft.irfft(f * np.conj(f), n=n, axis=0)[:T].mean(axis=1)
    acf /= np.arange(T, 0, -1)
    rho = acf / acf[0]
    tau = 1.0
    for M in range(1, T):
        tau += 2.0 * rho[M]
        if M >= c * tau:
            return float(tau), M
    return float(tau), T - 1


def mean_and_error(x, tau):
    """Mean of x[step][walker] and its standard error with the autocorrelation time."""
    x = np.asarray(x, dtype=np.float64)
    n_eff = x.size / max(tau, 1.0)
    return float(x.mean()), float(x.std() / np.sqrt(n_eff))
