"""CPU oracle of the surrogate-gradient adjoint — TEST INFRASTRUCTURE ONLY.

The differentiable form of the partitioned LIF step (no counterpart in the
paper, which simulates but does not train):

- populations: {excitatory, inhibitory} x {VN 0, VN 1, ...}: pop(j) =
  2 vn(j) + (0 if j is excitatory else 1);
- inputs: A_jb(t) = int32 sum of the weights of the synapses from population
  b that arrive at j at step t (the integer delivery of the plain step, kept
  per source population);
- current (fp32, fixed order, no FMA):
      I_j = (((G[a][0] A_j0 + G[a][1] A_j1) + G[a][2] A_j2) + G[a][3] A_j3)
            + w_ext (lam_a + sigma xi_j(t)),
  a = pop(j); G = population-pair gains, lam = drive rates (arrivals per
  step); xi_j(t) = (sum of 12 bytes of Philox4x32-10(counter (j, t, 0xAD, 0),
  key = seed) - 1530) / 256, an Irwin-Hall(12) approximation of N(0, 1) that
  both sides compute exactly;
- membrane as the plain step: V_pre = (E_L + alpha (V - E_L)) + I 2^-10,
  spike S = [V_pre >= theta], hard reset to V_reset and t_ref refractory
  steps (V held at V_reset, no spike);
- loss inputs: population rates r_a = sum_t sum_{j in a} S_j(t) / (T N_a).

Backward (surrogate gradient, reset detached): with gVpre the adjoint of
V_pre and gV that of V,
      gS_j(t)    = dL/dr_a / (T N_a) + 2^-10 sum_{j->k, delay d} G[pop k][a] w gVpre_k(t+d)
      gVpre_j(t) = gV_j(t) (1 - S_j(t)) + gS_j(t) / (1 + beta |V_pre_j(t) - theta|)^2
      gV_j(t-1)  = alpha gVpre_j(t)            (both 0 while j is refractory)
      dL/dG[a][b] = 2^-10 sum_t sum_{j in a} gVpre_j(t) A_jb(t)
      dL/dlam_a   = 2^-10 w_ext sum_t sum_{j in a} gVpre_j(t).
The sum over j's outgoing synapses is the transpose of the delivery.

The smooth variant (FP64 only, for finite differences): s = logistic(beta
(V_pre - theta)) in place of S, soft reset V = V_pre - (theta - V_reset) s,
no refractory, float inputs A_jb = sum w s; its backward is exact.

`forward_fp32` reproduces the GPU forward bit for bit (same operations in
float32); `backward` runs in float64 on a recorded trajectory.  Pinned in
tests/test_oracle_adjoint.py by finite differences (smooth) and by PyTorch
autograd of an unrolled graph (surrogate).
"""
from __future__ import annotations

import dataclasses

import numpy as np

NOISE_TAG = 0xAD
SIGMA = np.float32(0.9)
BETA = 5.0


# ---------------------------------------------------------------- Philox4x32-10
def philox_blocks(c0: np.ndarray, c1: int, c2: int, c3: int, k0: int, k1: int) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) of counters (c0[i], c1, c2, c3) and key
    (k0, k1), vectorised over c0: returns [n, 4] uint32."""
    m0, m1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    w0, w1 = 0x9E3779B9, 0xBB67AE85
    mask = np.uint64(0xFFFFFFFF)
    x0 = np.asarray(c0, np.uint64) & mask
    n = x0.shape[0]
    x1 = np.full(n, c1 & 0xFFFFFFFF, np.uint64)
    x2 = np.full(n, c2 & 0xFFFFFFFF, np.uint64)
    x3 = np.full(n, c3 & 0xFFFFFFFF, np.uint64)
    a, b = k0 & 0xFFFFFFFF, k1 & 0xFFFFFFFF
    for _ in range(10):
        p0 = m0 * x0
        p1 = m1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        y0 = hi1 ^ x1 ^ np.uint64(a)
        y2 = hi0 ^ x3 ^ np.uint64(b)
        x0, x1, x2, x3 = y0, lo1, y2, lo0
        a = (a + w0) & 0xFFFFFFFF
        b = (b + w1) & 0xFFFFFFFF
    return np.stack([x0, x1, x2, x3], axis=1).astype(np.uint32)


def noise(seed: int, M: int, t: int) -> np.ndarray:
    """xi_j(t) for j = 0..M-1 (float32, exact)."""
    w = philox_blocks(np.arange(M, dtype=np.uint64), t, NOISE_TAG, 0, seed & 0xFFFFFFFF, seed >> 32)
    bts = w[:, :3].view(np.uint8).reshape(M, 12).astype(np.int64).sum(axis=1)
    return ((bts - 1530).astype(np.float32) / np.float32(256.0)).astype(np.float32)


# ---------------------------------------------------------------- model
@dataclasses.dataclass
class AdjointNet:
    """A network in the adjoint form: the synapse list, populations and dynamics."""
    M: int
    syn_ptr: np.ndarray
    tgt: np.ndarray
    w: np.ndarray
    d: np.ndarray
    v0: np.ndarray
    pop: np.ndarray        # [M] population of each neuron
    n_pop: int
    e_l: float
    v_th: float
    v_reset: float
    alpha: np.float32
    t_ref: int
    w_ext: float
    seed: int
    dmax: int

    @property
    def src(self) -> np.ndarray:
        return np.repeat(np.arange(self.M, dtype=np.int64), np.diff(self.syn_ptr))

    def pop_sizes(self) -> np.ndarray:
        return np.bincount(self.pop, minlength=self.n_pop).astype(np.float64)


def populations(is_exc: np.ndarray, part: np.ndarray, vn_of_part: np.ndarray) -> np.ndarray:
    """pop(j) = 2 vn(j) + (0 excitatory, 1 inhibitory)."""
    return (2 * vn_of_part[part] + (1 - is_exc.astype(np.int64))).astype(np.int64)


def from_synth(g, dyn, part: np.ndarray, vn_of_part: np.ndarray, alpha: np.float32) -> AdjointNet:
    pop = populations(g.is_exc, part, vn_of_part)
    return AdjointNet(g.M, g.syn_ptr.astype(np.int64), g.tgt.astype(np.int64), g.w.astype(np.int64),
                      g.d.astype(np.int64), g.v0.astype(np.float32), pop, int(pop.max()) + 1,
                      dyn.e_l, dyn.v_th, dyn.v_reset, np.float32(alpha), dyn.t_ref, float(dyn.w_ext),
                      dyn.drive_seed, int(g.d.max()) if g.E else 1)


@dataclasses.dataclass
class Trajectory:
    vpre: np.ndarray   # [T, M] float32
    spk: np.ndarray    # [T, M] bool
    refr: np.ndarray   # [T, M] bool (refractory at the step: no update)
    A: np.ndarray      # [T, M, n_pop] int64
    rates: np.ndarray  # [n_pop]


def forward_fp32(net: AdjointNet, G: np.ndarray, lam: np.ndarray, T: int) -> Trajectory:
    """T steps from V = v0, ref = 0: the hard-threshold forward in float32."""
    f32 = np.float32
    G = np.asarray(G, f32).reshape(net.n_pop, net.n_pop)
    lam = np.asarray(lam, f32)
    M, npop = net.M, net.n_pop
    D = net.dmax + 1
    src = net.src
    spop = net.pop[src]
    ring = np.zeros((D, M, npop), np.int64)
    V = net.v0.copy()
    ref = np.zeros(M, np.int64)
    tr = Trajectory(np.zeros((T, M), f32), np.zeros((T, M), bool), np.zeros((T, M), bool),
                    np.zeros((T, M, npop), np.int64), np.zeros(npop))
    a = net.pop
    e_l, v_th, v_reset = f32(net.e_l), f32(net.v_th), f32(net.v_reset)
    for t in range(T):
        A = ring[t % D].copy()
        ring[t % D] = 0
        Af = A.astype(f32)
        Gr = G[a]  # [M, npop]
        irec = (Gr[:, 0] * Af[:, 0]).astype(f32)
        for b in range(1, npop):
            irec = (irec + Gr[:, b] * Af[:, b]).astype(f32)
        x1 = (SIGMA * noise(net.seed, M, t)).astype(f32)
        x2 = (lam[a] + x1).astype(f32)
        drv = (f32(net.w_ext) * x2).astype(f32)
        I = (irec + drv).astype(f32)
        refr = ref > 0
        u = (V - e_l).astype(f32)
        au = (net.alpha * u).astype(f32)
        vp = (e_l + au).astype(f32)
        vp = (vp + (I * f32(0.0009765625)).astype(f32)).astype(f32)
        S = (~refr) & (vp >= v_th)
        tr.vpre[t], tr.spk[t], tr.refr[t], tr.A[t] = vp, S, refr, A
        V = np.where(refr | S, v_reset, vp).astype(f32)
        ref = np.where(refr, ref - 1, np.where(S, net.t_ref, 0))
        # delivery of the step's spikes
        fired = np.nonzero(S)[0]
        if len(fired):
            idx = np.concatenate([np.arange(net.syn_ptr[i], net.syn_ptr[i + 1]) for i in fired])
            np.add.at(ring, ((t + net.d[idx]) % D, net.tgt[idx], spop[idx]), net.w[idx])
    tr.rates = np.bincount(a, weights=tr.spk.sum(axis=0), minlength=npop) / (T * net.pop_sizes())
    return tr


def _gather_tables(net: AdjointNet, G: np.ndarray):
    """Loop invariants of the gather: the synapses' sources, the products
    G[pop k][pop j] w (float64) and the position of each synapse's (delay,
    target) in a [D, M] table of adjoints indexed by delay."""
    src = net.src
    gw = G[net.pop[net.tgt], net.pop[src]] * net.w
    pos = net.d * net.M + net.tgt
    return src, gw, pos


def _gather(net: AdjointNet, tabs, ahead: np.ndarray) -> np.ndarray:
    """sum_{j->k, d} G[pop k][pop j] w gVpre_k(t+d) for every j (float64);
    ahead[d] holds gVpre(t+d) for d = 0..D-1 (tabs from _gather_tables)."""
    src, gw, pos = tabs
    val = gw * ahead.reshape(-1)[pos]
    return np.bincount(src, weights=val, minlength=net.M)


def backward(net: AdjointNet, G: np.ndarray, lam: np.ndarray, tr: Trajectory, grates: np.ndarray,
             smooth: bool = False, beta: float = BETA):
    """Gradients (dG [n_pop, n_pop], dlam [n_pop]) of a loss with dL/dr = grates,
    in float64, through the recorded trajectory `tr` (hard threshold with the
    surrogate, or the smooth variant)."""
    G = np.asarray(G, np.float64).reshape(net.n_pop, net.n_pop)
    T, M = tr.vpre.shape
    D = net.dmax + 1
    c = 2.0 ** -10
    a = net.pop
    direct = np.asarray(grates, np.float64)[a] / (T * net.pop_sizes()[a])
    # ahead[d] = gVpre(t + d) for the step t being processed (d = 0..D-1)
    ahead = np.zeros((D, M))
    tabs = _gather_tables(net, G)
    gV = np.zeros(M)
    dG = np.zeros_like(G)
    dlam = np.zeros(net.n_pop)
    theta = float(net.v_th)
    gap = float(net.v_th) - float(net.v_reset)
    for t in range(T - 1, -1, -1):
        ahead = np.roll(ahead, 1, axis=0)
        ahead[0] = 0.0
        gS = direct + c * _gather(net, tabs, ahead)
        x = tr.vpre[t].astype(np.float64) - theta
        if smooth:
            s = 1.0 / (1.0 + np.exp(-beta * x))
            ds = beta * s * (1.0 - s)
            gvp = gV * (1.0 - gap * ds) + gS * ds
        else:
            sg = 1.0 / (1.0 + beta * np.abs(x)) ** 2
            gvp = gV * (1.0 - tr.spk[t]) + gS * sg
            gvp = np.where(tr.refr[t], 0.0, gvp)
        ahead[0] = gvp
        gV = float(net.alpha) * gvp
        dG += c * np.stack([np.bincount(a, weights=gvp * tr.A[t][:, b], minlength=net.n_pop)
                            for b in range(net.n_pop)], axis=1)
        dlam += c * net.w_ext * np.bincount(a, weights=gvp, minlength=net.n_pop)
    return dG, dlam


def forward_smooth(net: AdjointNet, G: np.ndarray, lam: np.ndarray, T: int, beta: float = BETA) -> Trajectory:
    """The smooth variant in float64: logistic spikes, soft reset, no refractory."""
    G = np.asarray(G, np.float64).reshape(net.n_pop, net.n_pop)
    lam = np.asarray(lam, np.float64)
    M, npop = net.M, net.n_pop
    D = net.dmax + 1
    src = net.src
    spop = net.pop[src]
    ring = np.zeros((D, M, npop))
    V = net.v0.astype(np.float64)
    a = net.pop
    tr = Trajectory(np.zeros((T, M)), np.zeros((T, M)), np.zeros((T, M), bool), np.zeros((T, M, npop)),
                    np.zeros(npop))
    gap = net.v_th - net.v_reset
    for t in range(T):
        A = ring[t % D].copy()
        ring[t % D] = 0
        I = (G[a] * A).sum(axis=1) + net.w_ext * (lam[a] + float(SIGMA) * noise(net.seed, M, t).astype(np.float64))
        vp = net.e_l + float(net.alpha) * (V - net.e_l) + I * 2.0 ** -10
        s = 1.0 / (1.0 + np.exp(-beta * (vp - net.v_th)))
        tr.vpre[t], tr.spk[t], tr.A[t] = vp, s, A
        V = vp - gap * s
        np.add.at(ring, ((t + net.d) % D, net.tgt, spop), net.w * s[src])
    tr.rates = np.bincount(a, weights=tr.spk.sum(axis=0), minlength=npop) / (T * net.pop_sizes())
    return tr
