"""Seeded synthetic workloads shaped like the paper's benchmark families (Sec. 8.1).

This package only generates inputs: model definitions written with the pattern builder, their
data arrays, and evaluation points (x, y, sigma).  It holds none of the derivative arithmetic and is
shared by the oracle tests, the GPU parity tests, the smoke check and the benchmark.

Families (the paper's suites are not available; these stand in for them):
  * rosenbrock(n)        chained Rosenbrock objective with trig/exp equality constraints (an LV-style
                         instance, Sec. 8.1 "Luksan-Vlcek problems").
  * acopf(B, L, G, seed) polar AC optimal power flow with 15 patterns (Sec. 8.1 "PGLIB-OPF"; the
                         balance constraints use augmentations as in Sec. 3.3).
  * pde(N)               distributed control of -Lap u + u^3 = c on an N x N grid, 5-point stencil
                         (a COPS-style PDE-constrained instance).
  * acopf_batch(...)     many ACOPF instances of uneven size with per-instance load multipliers.
  * goddard(T)           Goddard rocket, trapezoidal discretisation with T steps (Eq. (rocket); a
                         COPS-style optimal-control instance with exp and division-heavy patterns).
  * two_stage_acopf(...) two-stage stochastic ACOPF (Eq. (extensions), B = 1): generator active
                         power is the shared first stage, voltages, reactive power and flows are
                         per scenario, and scenario loads are per-scenario parameters.
Every random number comes from numpy's PCG64 (`np.random.default_rng(seed)`).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from paper_2608_16265_gb300 import ir
from paper_2608_16265_gb300.ir import Model, TwoStageModel, sin, cos, exp


@dataclass
class Workload:
    name: str
    model: Model
    flat: ir.FlatModel
    meta: dict


# ------------------------------------------------------------------ Rosenbrock-type
def rosenbrock(n: int = 1000) -> Workload:
    """Objective  sum_{i=1}^{n-1} 100 (x_{i+1} - x_i^2)^2 + (1 - x_i)^2;
    constraints for i = 1..n-2:
      3 x_{i+1}^3 + 2 x_{i+2} - 5 + sin(x_{i+1} - x_{i+2}) sin(x_{i+1} + x_{i+2}) + 4 x_{i+1}
      - x_i exp(x_i - x_{i+1}) - 3 = 0.
    0-based: objective instance k uses x[k], x[k+1]; constraint instance k uses x[k..k+2]."""
    m = Model()
    x = m.add_var(n)
    m.add_obj(lambda d: 100 * (x[d.k + 1] - x[d.k] ** 2) ** 2 + (1 - x[d.k]) ** 2,
              n=n - 1, name="rosenbrock")
    m.add_con(lambda d: 3 * x[d.k + 1] ** 3 + 2 * x[d.k + 2] - 5
              + sin(x[d.k + 1] - x[d.k + 2]) * sin(x[d.k + 1] + x[d.k + 2])
              + 4 * x[d.k + 1] - x[d.k] * exp(x[d.k] - x[d.k + 1]) - 3,
              n=n - 2, name="trig_exp")
    return Workload(f"rosenbrock_n{n}", m, m.flat(), dict(n=n))


def rosenbrock_point(wl: Workload, seed: int):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, wl.flat.nvar)
    y = rng.standard_normal(wl.flat.ncon)
    return x, y, 1.0


# ------------------------------------------------------------------ AC optimal power flow (polar)
def _network(B: int, L: int, rng) -> np.ndarray:
    """Ring 0-1-...-(B-1)-0 plus L-B random chords without self-loops or repeated pairs."""
    if L < B:
        raise ValueError("need at least as many branches as buses (ring)")
    edges = [(i, (i + 1) % B) for i in range(B)]
    seen = {(min(a, b), max(a, b)) for a, b in edges}
    max_pairs = B * (B - 1) // 2
    if L > max_pairs:
        raise ValueError("too many branches for a simple graph")
    while len(edges) < L:
        need = L - len(edges)
        u = rng.integers(0, B, 2 * need + 8)
        v = rng.integers(0, B, 2 * need + 8)
        for a, b in zip(u.tolist(), v.tolist()):
            key = (min(a, b), max(a, b))
            if a == b or key in seen:
                continue
            seen.add(key)
            edges.append((a, b))
            if len(edges) == L:
                break
    return np.asarray(edges, dtype=np.int32)


def acopf(B: int, L: int, G: int, seed: int = 0, load_mult: float = 1.0,
          shunts: bool = False) -> Workload:
    """Polar ACOPF, 15 patterns.  Variables: va[B], vm[B], pg[G], qg[G], p[2L], q[2L] (arc a < L is
    the from end of branch a, arc L + a its to end).  Branch model: tap 1, no shift, series
    admittance g + jb = 1/(r + jx), line charging b_c split evenly between the ends.

    Distributions: r ~ U[0.001, 0.05], x ~ U[0.01, 0.3], b_c ~ U[0, 0.05]; Pd ~ U[0, 1] * load_mult,
    Qd = 0.3 Pd; c2 ~ U[0, 0.1], c1 ~ U[1, 50]; generators on uniformly drawn buses; reference bus =
    bus of generator 0.  Shunts gs, bs are zero unless `shunts` (then U[0, 0.05])."""
    rng = np.random.default_rng(seed)
    br = _network(B, L, rng)
    f, t = br[:, 0].copy(), br[:, 1].copy()
    r = rng.uniform(0.001, 0.05, L)
    xx = rng.uniform(0.01, 0.3, L)
    bc = rng.uniform(0.0, 0.05, L)
    z2 = r * r + xx * xx
    g, b = r / z2, -xx / z2
    gff = g.copy(); bff = b + bc / 2
    gft = -g; bft = -b.copy()
    gtt = g.copy(); btt = b + bc / 2
    gtf = -g; btf = -b.copy()
    pd = rng.uniform(0.0, 1.0, B) * load_mult
    qd = 0.3 * pd
    gs = rng.uniform(0.0, 0.05, B) if shunts else np.zeros(B)
    bs = rng.uniform(0.0, 0.05, B) if shunts else np.zeros(B)
    gbus = rng.integers(0, B, G).astype(np.int32)
    c2 = rng.uniform(0.0, 0.1, G)
    c1 = rng.uniform(1.0, 50.0, G)

    m = Model()
    va = m.add_var(B)
    vm = m.add_var(B)
    pg = m.add_var(G)
    qg = m.add_var(G)
    p = m.add_var(2 * L)
    q = m.add_var(2 * L)

    gens = dict(bus=gbus, c2=c2, c1=c1)
    m.add_obj(lambda d: d.c2 * pg[d.k] ** 2 + d.c1 * pg[d.k], data=gens, name="gen_cost")
    m.add_con(lambda d: va[d.ref], data=dict(ref=np.array([gbus[0]], np.int32)), name="ref_angle")
    brd = dict(f=f, t=t, gff=gff, bff=bff, gft=gft, bft=bft, gtt=gtt, btt=btt, gtf=gtf, btf=btf)
    m.add_con(lambda d: p[d.k] - (d.gff * vm[d.f] ** 2 + vm[d.f] * vm[d.t] * (
        d.gft * cos(va[d.f] - va[d.t]) + d.bft * sin(va[d.f] - va[d.t]))), data=brd, name="p_from")
    m.add_con(lambda d: q[d.k] - (-d.bff * vm[d.f] ** 2 - vm[d.f] * vm[d.t] * (
        d.bft * cos(va[d.f] - va[d.t]) - d.gft * sin(va[d.f] - va[d.t]))), data=brd, name="q_from")
    m.add_con(lambda d: p[d.k + L] - (d.gtt * vm[d.t] ** 2 + vm[d.t] * vm[d.f] * (
        d.gtf * cos(va[d.t] - va[d.f]) + d.btf * sin(va[d.t] - va[d.f]))), data=brd, name="p_to")
    m.add_con(lambda d: q[d.k + L] - (-d.btt * vm[d.t] ** 2 - vm[d.t] * vm[d.f] * (
        d.btf * cos(va[d.t] - va[d.f]) - d.gtf * sin(va[d.t] - va[d.f]))), data=brd, name="q_to")
    m.add_con(lambda d: va[d.f] - va[d.t], data=dict(f=f, t=t), name="angle_diff")
    m.add_con(lambda d: p[d.k] ** 2 + q[d.k] ** 2, n=L, name="thermal_from")
    m.add_con(lambda d: p[d.k + L] ** 2 + q[d.k + L] ** 2, n=L, name="thermal_to")
    busd = dict(pd=pd, qd=qd, gs=gs, bs=bs)
    cp = m.add_con(lambda d: d.pd + d.gs * vm[d.k] ** 2, data=busd, name="p_balance")
    cq = m.add_con(lambda d: d.qd - d.bs * vm[d.k] ** 2, data=busd, name="q_balance")
    m.add_con_aug(cp, lambda d: (d.bus, -pg[d.k]), data=dict(bus=gbus), name="gen_p")
    m.add_con_aug(cq, lambda d: (d.bus, -qg[d.k]), data=dict(bus=gbus), name="gen_q")
    arc_bus = np.concatenate([f, t]).astype(np.int32)
    m.add_con_aug(cp, lambda d: (d.bus, p[d.k]), data=dict(bus=arc_bus), name="arc_p")
    m.add_con_aug(cq, lambda d: (d.bus, q[d.k]), data=dict(bus=arc_bus), name="arc_q")
    meta = dict(B=B, L=L, G=G, seed=seed, load_mult=load_mult)
    return Workload(f"acopf_b{B}_l{L}_g{G}", m, m.flat(), meta)


def acopf_point(wl: Workload, seed: int):
    """Flat start (vm = 1, everything else 0) plus 0.05 N(0,1) on every variable;
    y ~ N(0, 1); sigma = 1."""
    rng = np.random.default_rng(seed)
    B = wl.meta["B"]
    x = np.zeros(wl.flat.nvar)
    x[B:2 * B] = 1.0
    x += 0.05 * rng.standard_normal(wl.flat.nvar)
    y = rng.standard_normal(wl.flat.ncon)
    return x, y, 1.0


# ------------------------------------------------------------------ PDE-constrained control
def pde(N: int = 1000) -> Workload:
    """min 0.5 ||u - u_d||^2 + 1e-4 * 0.5 ||c||^2  s.t.  (4u_ij - sum of 4 neighbours)/h^2 + u_ij^3
    - c_ij = 0 at interior nodes, h = 1/(N-1), u_d = sin(pi x) sin(pi y).  u lives on all N^2 nodes
    (boundary values fixed by bounds, which do not enter derivatives), c on the (N-2)^2 interior."""
    h = 1.0 / (N - 1)
    ih2 = 1.0 / (h * h)
    m = Model()
    u = m.add_var(N, N)
    c = m.add_var(N - 2, N - 2)
    ii, jj = np.meshgrid(np.arange(1, N - 1, dtype=np.int32), np.arange(1, N - 1, dtype=np.int32),
                         indexing="ij")
    interior = dict(i=ii.ravel(), j=jj.ravel())
    gx = np.arange(N) * h
    ud = (np.sin(np.pi * gx)[:, None] * np.sin(np.pi * gx)[None, :]).ravel()
    m.add_obj(lambda d: 0.5 * (u.at(d.k) - d.ud) ** 2, data=dict(ud=ud), name="track")
    m.add_obj(lambda d: 0.5e-4 * c.at(d.k) ** 2, n=(N - 2) * (N - 2), name="control")
    m.add_con(lambda d: (4 * u[d.i, d.j] - u[d.i - 1, d.j] - u[d.i + 1, d.j] - u[d.i, d.j - 1]
                         - u[d.i, d.j + 1]) * ih2 + u[d.i, d.j] ** 3 - c[d.i - 1, d.j - 1],
              data=interior, name="state")
    return Workload(f"pde_n{N}", m, m.flat(), dict(N=N))


def pde_point(wl: Workload, seed: int):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, wl.flat.nvar)
    y = rng.standard_normal(wl.flat.ncon)
    return x, y, 1.0


# ------------------------------------------------------------------ batch of uneven ACOPF instances
def acopf_batch_sizes(n_inst: int = 256, seed: int = 7, bmin: int = 200, bmax: int = 20000):
    """Buses ~ log-uniform[bmin, bmax], branches = 1.5 x buses, generators = buses / 6,
    load multiplier ~ U[0.8, 1.2]; one row per instance: (B, L, G, seed, load_mult)."""
    rng = np.random.default_rng(seed)
    B = np.exp(rng.uniform(math.log(bmin), math.log(bmax), n_inst)).astype(np.int64)
    B = np.maximum(B, 3)
    L = (1.5 * B).astype(np.int64)
    G = np.maximum(B // 6, 1)
    mult = rng.uniform(0.8, 1.2, n_inst)
    seeds = rng.integers(0, 2 ** 31 - 1, n_inst)
    return [(int(b), int(l), int(g), int(s), float(mu)) for b, l, g, s, mu in zip(B, L, G, seeds, mult)]


def acopf_batch(n_inst: int = 256, seed: int = 7, bmin: int = 200, bmax: int = 20000) -> List[Workload]:
    return [acopf(b, l, g, seed=s, load_mult=mu)
            for (b, l, g, s, mu) in acopf_batch_sizes(n_inst, seed, bmin, bmax)]


# ------------------------------------------------------------------ two-stage stochastic ACOPF
def two_stage_acopf(B: int, L: int, G: int, S: int, seed: int = 0, spread: float = 0.1) -> Workload:
    """ACOPF of `acopf` in two stages over S load scenarios.  Root (shared) variables: pg[G].
    Per-scenario variables: va, vm[B], qg[G], p, q[2L].  Per-scenario parameters: pd, qd[B]
    (scenario s: the base loads times (1 + spread N(0,1)) per bus).  Objective: the root generation
    cost plus, per scenario, (1/S) 0.01 qg^2.  Per scenario: the reference angle, the four flow
    definitions, angle difference, two thermal limits, P and Q balances with the generator (root
    pg, scenario qg) and arc augmentations.  Network and branch data as in `acopf`."""
    rng = np.random.default_rng(seed)
    br = _network(B, L, rng)
    f, t = br[:, 0].astype(np.int32), br[:, 1].astype(np.int32)
    r = rng.uniform(0.001, 0.05, L)
    xx = rng.uniform(0.01, 0.3, L)
    bc = rng.uniform(0.0, 0.05, L)
    z2 = r * r + xx * xx
    g, b = r / z2, -xx / z2
    gff, bff, gft, bft = g.copy(), b + bc / 2, -g, -b.copy()
    gtt, btt, gtf, btf = g.copy(), b + bc / 2, -g, -b.copy()
    pd0 = rng.uniform(0.0, 1.0, B)
    gbus = rng.integers(0, B, G).astype(np.int32)
    c2 = rng.uniform(0.0, 0.1, G)
    c1 = rng.uniform(1.0, 50.0, G)
    pd = pd0[:, None] * (1.0 + spread * rng.standard_normal((B, S)))
    qd = 0.3 * pd

    m = TwoStageModel(S)
    pg = m.add_var(G)
    va = m.add_var(B, scenario=True)
    vm = m.add_var(B, scenario=True)
    qg = m.add_var(G, scenario=True)
    p = m.add_var(2 * L, scenario=True)
    q = m.add_var(2 * L, scenario=True)
    PD = m.add_par(pd, scenario=True)
    QD = m.add_par(qd, scenario=True)

    gi = np.arange(G, dtype=np.int32)
    m.add_obj(lambda d: d.c2 * pg[d.k] ** 2 + d.c1 * pg[d.k], data=dict(c2=c2, c1=c1), name="gen_cost")
    m.add_obj(lambda d: (0.01 / S) * qg[d.g, d.s] ** 2, data=dict(g=gi), scenario=True, name="q_cost")
    m.add_con(lambda d: va[d.ref, d.s], data=dict(ref=np.array([gbus[0]], np.int32)), scenario=True,
              name="ref_angle")
    brd = dict(a=np.arange(L, dtype=np.int32), f=f, t=t, gff=gff, bff=bff, gft=gft, bft=bft, gtt=gtt,
               btt=btt, gtf=gtf, btf=btf)

    def th(d, i, j):
        return va[i, d.s] - va[j, d.s]

    m.add_con(lambda d: p[d.a, d.s] - (d.gff * vm[d.f, d.s] ** 2 + vm[d.f, d.s] * vm[d.t, d.s] * (
        d.gft * cos(th(d, d.f, d.t)) + d.bft * sin(th(d, d.f, d.t)))), data=brd, scenario=True, name="p_from")
    m.add_con(lambda d: q[d.a, d.s] - (-d.bff * vm[d.f, d.s] ** 2 - vm[d.f, d.s] * vm[d.t, d.s] * (
        d.bft * cos(th(d, d.f, d.t)) - d.gft * sin(th(d, d.f, d.t)))), data=brd, scenario=True, name="q_from")
    m.add_con(lambda d: p[d.a + L, d.s] - (d.gtt * vm[d.t, d.s] ** 2 + vm[d.t, d.s] * vm[d.f, d.s] * (
        d.gtf * cos(th(d, d.t, d.f)) + d.btf * sin(th(d, d.t, d.f)))), data=brd, scenario=True, name="p_to")
    m.add_con(lambda d: q[d.a + L, d.s] - (-d.btt * vm[d.t, d.s] ** 2 - vm[d.t, d.s] * vm[d.f, d.s] * (
        d.btf * cos(th(d, d.t, d.f)) - d.gtf * sin(th(d, d.t, d.f)))), data=brd, scenario=True, name="q_to")
    m.add_con(lambda d: va[d.f, d.s] - va[d.t, d.s], data=dict(f=f, t=t), scenario=True, name="angle_diff")
    ai = dict(a=np.arange(L, dtype=np.int32))
    m.add_con(lambda d: p[d.a, d.s] ** 2 + q[d.a, d.s] ** 2, data=ai, scenario=True, name="thermal_from")
    m.add_con(lambda d: p[d.a + L, d.s] ** 2 + q[d.a + L, d.s] ** 2, data=ai, scenario=True, name="thermal_to")
    bi = dict(i=np.arange(B, dtype=np.int32))
    cp = m.add_con(lambda d: PD[d.i, d.s], data=bi, scenario=True, name="p_balance")
    cq = m.add_con(lambda d: QD[d.i, d.s], data=bi, scenario=True, name="q_balance")
    m.add_con_aug(cp, lambda d: (d.bus, -pg[d.g]), data=dict(bus=gbus, g=gi), scenario=True, name="gen_p")
    m.add_con_aug(cq, lambda d: (d.bus, -qg[d.g, d.s]), data=dict(bus=gbus, g=gi), scenario=True, name="gen_q")
    arcs = dict(bus=np.concatenate([f, t]).astype(np.int32), a=np.arange(2 * L, dtype=np.int32))
    m.add_con_aug(cp, lambda d: (d.bus, p[d.a, d.s]), data=arcs, scenario=True, name="arc_p")
    m.add_con_aug(cq, lambda d: (d.bus, q[d.a, d.s]), data=arcs, scenario=True, name="arc_q")
    meta = dict(B=B, L=L, G=G, S=S, seed=seed, spread=spread, vm=vm, pd=PD, qd=QD)
    return Workload(f"two_stage_acopf_b{B}_l{L}_g{G}_s{S}", m, m.flat(), meta)


def two_stage_point(wl: Workload, seed: int):
    """vm = 1 in every scenario, everything else 0, plus 0.05 N(0,1) on every variable;
    y ~ N(0, 1); sigma = 1."""
    rng = np.random.default_rng(seed)
    x = np.zeros(wl.flat.nvar)
    vm = wl.meta["vm"]
    for s in range(wl.meta["S"]):
        x[vm.scenario_range(s)] = 1.0
    x += 0.05 * rng.standard_normal(wl.flat.nvar)
    y = rng.standard_normal(wl.flat.ncon)
    return x, y, 1.0


# ------------------------------------------------------------------ Goddard rocket (optimal control)
GODDARD = dict(h0=1.0, v0=0.0, m0=1.0, g0=1.0, Tc=3.5, hc=500.0, vc=620.0, mc=0.6)


def goddard(T: int = 1000) -> Workload:
    """Eq. (rocket) with T trapezoidal steps; variables h, v, m, tau on t = 0..T and the step dt.
    Drag D(h, v) = Dc v^2 exp(-hc (h - h0)/h0), gravity g(h) = g0 (h0/h)^2, exhaust velocity
    c = sqrt(g0 h0)/2, Dc = vc m0/(2 g0), final mass mf = mc m0 (a parameter).  The objective is the
    final altitude, written as minimising -h_T."""
    k = GODDARD
    c = 0.5 * math.sqrt(k["g0"] * k["h0"])
    Dc = 0.5 * k["vc"] * k["m0"] / k["g0"]
    m = Model()
    h = m.add_var(T + 1)
    v = m.add_var(T + 1)
    ms = m.add_var(T + 1)
    tau = m.add_var(T + 1)
    dt = m.add_var(1)
    mf = m.add_par([k["mc"] * k["m0"]])

    def accel(t):  # (tau - D)/m - g at step t
        drag = Dc * v[t] ** 2 * exp(-k["hc"] * (h[t] - k["h0"]) / k["h0"])
        return (tau[t] - drag) / ms[t] - k["g0"] * (k["h0"] / h[t]) ** 2

    m.add_obj(lambda d: -h[T], n=1, name="final_altitude")
    m.add_con(lambda d: h[d.k + 1] - h[d.k] - 0.5 * dt[0] * (v[d.k + 1] + v[d.k]), n=T, name="altitude")
    m.add_con(lambda d: v[d.k + 1] - v[d.k] - 0.5 * dt[0] * (accel(d.k + 1) + accel(d.k)), n=T, name="velocity")
    m.add_con(lambda d: ms[d.k + 1] - ms[d.k] + 0.5 * dt[0] * (tau[d.k + 1] + tau[d.k]) / c, n=T, name="mass")
    m.add_con(lambda d: h[0] - k["h0"], n=1, name="h_initial")
    m.add_con(lambda d: v[0] - k["v0"], n=1, name="v_initial")
    m.add_con(lambda d: ms[0] - k["m0"], n=1, name="m_initial")
    m.add_con(lambda d: ms[T] - mf[0], n=1, name="m_final")
    return Workload(f"goddard_T{T}", m, m.flat(), dict(T=T))


def goddard_point(wl: Workload, seed: int):
    """Around the usual starting trajectory: h = 1, v = s(1 - s), m from m0 to mf, tau = Tmax/2,
    dt = 1/T (s = t/T), each perturbed by 1 %; y ~ N(0, 1); sigma = 1."""
    rng = np.random.default_rng(seed)
    k = GODDARD
    T = wl.meta["T"]
    sgrid = np.arange(T + 1) / T
    mfin = k["mc"] * k["m0"]
    tmax = k["Tc"] * k["m0"] * k["g0"]
    x = np.concatenate([np.ones(T + 1), sgrid * (1 - sgrid), (mfin - k["m0"]) * sgrid + k["m0"],
                        np.full(T + 1, tmax / 2), [1.0 / T]])
    x *= 1 + 0.01 * rng.standard_normal(len(x))
    y = rng.standard_normal(wl.flat.ncon)
    return x, y, 1.0


# ------------------------------------------------------------------ named configurations
def config(name: str):
    """The benchmark configurations: returns (workloads, point function)."""
    if name == "rosenbrock":
        return [rosenbrock(1000)], rosenbrock_point
    if name == "acopf_small":
        return [acopf(500, 700, 100, seed=1)], acopf_point
    if name == "acopf_large":
        return [acopf(30000, 45000, 5000, seed=2)], acopf_point
    if name == "pde":
        return [pde(1000)], pde_point
    if name == "acopf_batch":
        return acopf_batch(256), acopf_point
    if name == "goddard":
        return [goddard(100000)], goddard_point
    raise KeyError(name)
