"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each ``pin_*`` function takes an oracle library handle (the real one, or a
copy with a planted mistake) and returns a list of failure strings (empty =
pass).  None of them re-types the oracle's own formula: each checks a
different statement of the same fact -- a moment identity, an alternative
form the paper prints, an exact Taylor identity, a conservation law, a
closed-form decay, a theory curve, or a number printed in the paper.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import theory as th
from paper_1204_4098_gb300 import inputs

EX, EY, Q = oracle.EX, oracle.EY, oracle.Q
CS2 = 1.0 / 3.0


def _close(name, got, want, rtol=0.0, atol=0.0):
    got, want = np.asarray(got, float), np.asarray(want, float)
    if not np.all(np.isfinite(got)) or not np.allclose(got, want, rtol=rtol, atol=atol):
        err = np.max(np.abs(got - want)) if got.shape == want.shape else "shape"
        return [f"{name}: got {got.ravel()[:6]} want {want.ravel()[:6]} (max err {err})"]
    return []


def _random_cell(rng, rho=None, u=0.05):
    """Random pre-collision populations near equilibrium."""
    rho = rng.uniform(0.05, 0.4) if rho is None else rho
    ux, uy = rng.uniform(-u, u, 2)
    f = oracle.feq(rho, ux, uy) * (1.0 + 0.05 * rng.uniform(-1, 1, Q))
    return f


# ---------------------------------------------------------------------------
# Eq. 2: equilibrium and weights
# ---------------------------------------------------------------------------

def pin_feq_moments(lib):
    """Eq. 2 has moments rho, rho u and rho c_s^2 I + rho u u (D2Q9, c_s^2=1/3),
    and at u = 0 returns the weights 4/9, 1/9 (x4), 1/36 (x4) (text after Eq. 2)."""
    fails = []
    rng = np.random.default_rng(10)
    fails += _close("weights", oracle.feq(1.0, 0.0, 0.0, lib=lib),
                    [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=1e-16)
    for _ in range(5):
        rho, ux, uy = rng.uniform(0.05, 0.5), *rng.uniform(-0.1, 0.1, 2)
        f = oracle.feq(rho, ux, uy, lib=lib)
        fails += _close("sum feq", f.sum(), rho, rtol=1e-14)
        fails += _close("sum feq e", [f @ EX, f @ EY], [rho * ux, rho * uy], atol=1e-15)
        Pi = np.array([[f @ (EX * EX), f @ (EX * EY)], [f @ (EY * EX), f @ (EY * EY)]])
        want = rho * CS2 * np.eye(2) + rho * np.outer([ux, uy], [ux, uy])
        fails += _close("sum feq ee", Pi, want, atol=1e-15)
    return fails


# ---------------------------------------------------------------------------
# Eq. 3: the interaction-force stencil
# ---------------------------------------------------------------------------

def pin_force_stencil_taylor(lib):
    """Eq. 3 with w(1) = 1/3, w(2) = 1/12: for a cubic polynomial psi the
    Taylor series of sum_a w psi(x+e_a) e_a terminates, and the isotropy of
    the weights (sum w e e = I, sum w e e e e = (1/3)(dd+dd+dd)) gives exactly
    grad psi + (1/6) grad lap psi.  So F = -G psi (grad psi + grad lap psi / 6)
    at every cell away from the periodic seam."""
    nx = ny = 16
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    x0, y0 = x - 7.3, y - 8.1
    psi = 2.0 + 0.1 * x0 - 0.05 * y0 + 0.01 * x0 * y0 + 0.003 * x0 ** 2 \
        + 0.002 * x0 ** 3 - 0.001 * x0 * y0 ** 2 + 0.0015 * y0 ** 3
    gx = 0.1 + 0.01 * y0 + 0.006 * x0 + 0.006 * x0 ** 2 - 0.001 * y0 ** 2
    gy = -0.05 + 0.01 * x0 - 0.002 * x0 * y0 + 0.0045 * y0 ** 2
    # lap psi = 0.006 + 0.012 x0 - 0.002 x0 + 0.009 y0
    lgx, lgy = 0.010, 0.009
    G = -1.0
    Fx, Fy = oracle.force(psi, G=G, lib=lib)
    inner = (slice(2, ny - 2), slice(2, nx - 2))
    fails = _close("Fx", Fx[inner], (-G * psi * (gx + lgx / 6.0))[inner], atol=1e-13)
    fails += _close("Fy", Fy[inner], (-G * psi * (gy + lgy / 6.0))[inner], atol=1e-13)
    return fails


def pin_force_pair_antisymmetry(lib):
    """Eq. 3 pairs x and x+e with opposite e, so the total force on a periodic
    domain vanishes for any psi field."""
    rng = np.random.default_rng(3)
    psi = rng.uniform(0.1, 0.5, (7, 5))
    Fx, Fy = oracle.force(psi, lib=lib)
    return _close("sum F", [Fx.sum(), Fy.sum()], [0.0, 0.0], atol=1e-15)


# ---------------------------------------------------------------------------
# Eq. 1: streaming
# ---------------------------------------------------------------------------

def pin_stream_moves_along_e(lib):
    """Eq. 1 left side: f_a leaves x and arrives at x + e_a (periodic)."""
    fails = []
    nx, ny = 5, 4
    for a in range(Q):
        f = np.zeros((Q, ny, nx))
        f[a, 0, 4] = 1.0
        out = oracle.stream(f, lib=lib)
        want = np.zeros_like(f)
        want[a, (0 + EY[a]) % ny, (4 + EX[a]) % nx] = 1.0
        fails += _close(f"stream a={a}", out, want, atol=0)
    return fails


# ---------------------------------------------------------------------------
# Table I and Eqs. 12-16, 31: forcing terms by their moments
# ---------------------------------------------------------------------------

def _forcing_term(lib, scheme, tau, sigma, f, Fx, Fy, psi, ueq):
    """F_a implied by a collision: f* - [f - (f - f_eq(rho, u_eq))/tau]."""
    rho = f.sum()
    post = oracle.collide_cell(scheme, tau, sigma, f, Fx, Fy, psi, lib=lib)
    return post - (f - (f - oracle.feq(rho, *ueq, lib=lib)) / tau)


def pin_table1_forcing_moments(lib):
    """Table I: every scheme is BGK towards f_eq(rho, u_eq) plus Guo's general
    forcing term (Eq. 12) with B = B_e F and C = C_e (v F + F v).  Guo's term
    has zeroth moment 0, first moment B_e F and second moment C (the D2Q9
    fourth-order isotropy), so each scheme is pinned by the velocity it puts in
    f_eq, the velocity in F_a and (B_e, C_e) of its Table I row."""
    fails = []
    rng = np.random.default_rng(7)
    for trial in range(4):
        f = _random_cell(rng)
        rho = f.sum()
        u = np.array([f @ EX, f @ EY]) / rho
        F = rng.uniform(-2e-3, 2e-3, 2)
        psi = rng.uniform(0.2, 0.5)
        for tau in (0.6, 0.8, 1.0, 1.7):
            sigma = 0.105
            v = u + F / (2 * rho)
            vprime = v + sigma * F / ((tau - 0.5) * psi ** 2)
            rows = {
                "SC": (oracle.SC, 0.0, u, u + tau * F / (2 * rho), 1.0, 1.0),
                "EDM": (oracle.EDM, 0.0, u, v, 1.0, 1.0),
                "Ladd": (oracle.LADD, 0.0, u, u, 1.0, 1.0),
                "Guo": (oracle.IMPROVED, 0.0, v, v, 1 - 1 / (2 * tau), 1 - 1 / (2 * tau)),
                "improved": (oracle.IMPROVED, sigma, v, vprime, 1 - 1 / (2 * tau), 1 - 1 / (2 * tau)),
                "EDM C_e=1/tau": (oracle.EDM_MOD, 0.0, u, v, 1.0, 1.0 / tau),
            }
            for name, (sch, sig, ueq, vbar, Be, Ce) in rows.items():
                Fa = _forcing_term(lib, sch, tau, sig, f, F[0], F[1], psi, ueq)
                C = Ce * (np.outer(vbar, F) + np.outer(F, vbar))
                M2 = np.array([[Fa @ (EX * EX), Fa @ (EX * EY)],
                               [Fa @ (EY * EX), Fa @ (EY * EY)]])
                tag = f"{name} tau={tau}"
                fails += _close(tag + " sum F_a", Fa.sum(), 0.0, atol=1e-15)
                fails += _close(tag + " sum F_a e", [Fa @ EX, Fa @ EY], Be * F, atol=1e-15)
                fails += _close(tag + " sum F_a ee", M2, C, atol=1e-15)
    return fails


def _guo_tensor_form(tau_factor, F, vbar, a):
    """First line of Eq. 31 / Eq. 12 written with explicit 2x2 tensors."""
    e = np.array([EX[a], EY[a]], float)
    w = oracle.W[a]
    C = np.outer(vbar, F) + np.outer(F, vbar)
    A = np.outer(e, e) - CS2 * np.eye(2)
    return w * tau_factor * (F @ e / CS2 + np.sum(C * A) / (2 * CS2 ** 2))


def pin_paper_rewrites(lib):
    """Eqs. 14-15: Shan-Chen = BGK to f_eq(rho,u) + F_SC with v_SC = u + tau F/(2 rho);
    Eq. 16: EDM = BGK to f_eq(rho,u) + F_EDM with v_EDM = u + F/(2 rho);
    Eq. 31: its two printed lines agree (tensor form vs vector form);
    text after Eq. 31: sigma = 0 is Guo's scheme (Eqs. 12-13);
    text before Eq. 17: Shan-Chen and EDM coincide at tau = 1."""
    fails = []
    rng = np.random.default_rng(11)
    for _ in range(4):
        f = _random_cell(rng)
        rho = f.sum()
        u = np.array([f @ EX, f @ EY]) / rho
        F = rng.uniform(-3e-3, 3e-3, 2)
        psi = rng.uniform(0.2, 0.5)
        for tau in (0.55, 0.7, 1.0, 1.3):
            bgk_u = f - (f - oracle.feq(rho, *u, lib=lib)) / tau
            v = u + F / (2 * rho)
            bgk_v = f - (f - oracle.feq(rho, *v, lib=lib)) / tau
            vsc = u + tau * F / (2 * rho)
            want_sc = bgk_u + np.array([_guo_tensor_form(1.0, F, vsc, a) for a in range(Q)])
            want_edm = bgk_u + np.array([_guo_tensor_form(1.0, F, v, a) for a in range(Q)])
            for sigma in (0.0, 0.0625, 0.125):
                vp = v + sigma * F / ((tau - 0.5) * psi ** 2)
                want_imp = bgk_v + np.array([_guo_tensor_form(1 - 1 / (2 * tau), F, vp, a)
                                             for a in range(Q)])
                got = oracle.collide_cell(oracle.IMPROVED, tau, sigma, f, *F, psi, lib=lib)
                fails += _close(f"Eq31 sigma={sigma} tau={tau}", got, want_imp, atol=1e-15)
            got_sc = oracle.collide_cell(oracle.SC, tau, 0.0, f, *F, psi, lib=lib)
            got_edm = oracle.collide_cell(oracle.EDM, tau, 0.0, f, *F, psi, lib=lib)
            fails += _close(f"Eq15 tau={tau}", got_sc, want_sc, atol=1e-15)
            fails += _close(f"Eq16 tau={tau}", got_edm, want_edm, atol=1e-15)
            if tau == 1.0:
                fails += _close("SC==EDM at tau=1", got_sc, got_edm, atol=1e-15)
    return fails


def pin_collision_momentum(lib):
    """Every forced scheme adds exactly F to the momentum in a collision
    (post-collision sum f* e = rho u + F, delta_t = 1), and none changes the
    mass; NOFORCE conserves both."""
    fails = []
    rng = np.random.default_rng(5)
    for _ in range(4):
        f = _random_cell(rng)
        rho = f.sum()
        j = np.array([f @ EX, f @ EY])
        F = rng.uniform(-3e-3, 3e-3, 2)
        for sch in (oracle.SC, oracle.EDM, oracle.IMPROVED, oracle.EDM_MOD, oracle.LADD):
            post = oracle.collide_cell(sch, 0.8, 0.1, f, *F, 0.3, lib=lib)
            fails += _close(f"mass s={sch}", post.sum(), rho, rtol=1e-15)
            fails += _close(f"momentum s={sch}", [post @ EX, post @ EY], j + F, atol=1e-15)
        post = oracle.collide_cell(oracle.NOFORCE, 0.8, 0.0, f, *F, 0.3, lib=lib)
        fails += _close("noforce momentum", [post @ EX, post @ EY], j, atol=1e-15)
    return fails


# ---------------------------------------------------------------------------
# Eqs. 8 and 23: equation of state and potential
# ---------------------------------------------------------------------------

def pin_eos_and_psi(lib):
    """The oracle's p_EOS equals Eq. 23 evaluated independently (theory tool,
    itself pinned by the critical point), psi reproduces p through the model
    EOS of Eq. 5 (p = rho c_s^2 + G psi^2 / 2), and densities outside the
    domain of psi are rejected rather than clamped."""
    fails = []
    T = th.temperature(0.8)
    eos = th.CarnahanStarling(T)
    for rho in (0.01, 0.1, 0.3, 0.45):
        fails += _close(f"p({rho})", oracle.p_eos(rho, T, lib=lib), eos.p(rho), rtol=1e-14)
        ps = oracle.psi(rho, T, lib=lib)
        fails += _close(f"Eq5 at {rho}", rho * CS2 + 0.5 * (-1.0) * ps ** 2, eos.p(rho),
                        rtol=1e-13, atol=1e-16)
    for bad in (0.0, -0.1, 1.0, 0.9, float("nan")):
        if oracle.psi(bad, T, lib=lib) is not None:
            fails.append(f"psi({bad}) accepted")
    return fails


# ---------------------------------------------------------------------------
# whole steps: conservation, fixed points, decay rates
# ---------------------------------------------------------------------------

def _lattice(lib, nx, ny, t=0.8):
    return oracle.Lattice(nx, ny, t, lib=lib)


def pin_step_conservation(lib):
    """Streaming permutes populations and every collision conserves mass and
    adds F, whose domain sum vanishes (Eq. 3): total mass and total momentum of
    a periodic domain are invariants of the step, for every scheme."""
    fails = []
    eos = th.CarnahanStarling(th.temperature(0.9))
    rg, rl, _ = th.maxwell(eos)
    rho0 = inputs.droplet(12, 10, rg, rl, 3.0, W=3.0)
    for sch, tau, sig in ((oracle.SC, 0.8, 0), (oracle.EDM, 0.7, 0),
                          (oracle.IMPROVED, 0.9, 0.105), (oracle.NOFORCE, 0.6, 0),
                          (oracle.EDM_MOD, 0.8, 0), (oracle.LADD, 1.2, 0)):
        lat = _lattice(lib, 12, 10, 0.9)
        lat.init_density(rho0)
        m0 = lat.mass()
        # the mass of f_eq(rho, 0) is the sum of the densities (sum_a w_a = 1)
        fails += _close("mass of the initial state", m0, float(np.sum(rho0)), rtol=1e-14)
        rc, _ = lat.step(200, sch, tau, sig)
        if rc:
            fails.append(f"scheme {sch} diverged")
            continue
        f = lat.f
        fails += _close(f"mass s={sch}", lat.mass(), m0, rtol=1e-13)
        mom = [np.sum(f * EX[:, None, None]), np.sum(f * EY[:, None, None])]
        fails += _close(f"momentum s={sch}", mom, [0, 0], atol=1e-14)
    return fails


def pin_uniform_fixed_point(lib):
    """A uniform density at rest has F = 0 (sum w e = 0) and f = f_eq, so it is
    a fixed point of every scheme; a uniform flow keeps its velocity."""
    fails = []
    for sch in (oracle.SC, oracle.EDM, oracle.IMPROVED):
        lat = _lattice(lib, 6, 5)
        rho = np.full((5, 6), 0.2)
        lat.init_density(rho)
        f0 = lat.f.copy()
        lat.step(10, sch, 0.7, 0.1)
        fails += _close(f"rest s={sch}", lat.f, f0, atol=1e-16)
        lat.init_density(rho, np.full((5, 6), 0.02), np.full((5, 6), -0.01))
        lat.step(10, sch, 0.7, 0.1)
        r, vx, vy = lat.observe()
        fails += _close(f"flow s={sch}", [vx.mean(), vy.mean(), np.ptp(r)], [0.02, -0.01, 0],
                        atol=1e-15)
    return fails


def _decay_rate(lib, n, tau, steps=400):
    rho, ux, uy, k = inputs.shear_wave(4, n, u0=1e-4, rho0=0.2)
    lat = _lattice(lib, 4, n, 1.5)
    lat.init_density(rho, ux, uy)
    amp = []
    for _ in range(2):
        lat.step(steps // 2, oracle.NOFORCE, tau)
        _, vx, _ = lat.observe(noforce=True)
        amp.append(np.sum(vx[:, 0] * np.sin(k * np.arange(n))) * 2 / n)
    rate = -np.log(amp[1] / amp[0]) / (steps // 2)
    return rate, (tau - 0.5) / 3.0 * k ** 2


def pin_shear_wave_decay(lib):
    """Force-free BGK (F = 0) is a Navier-Stokes solver with nu = c_s^2(tau - 1/2):
    a shear wave u_x = u0 sin(k y) decays as exp(-nu k^2 t).  The measured rate
    is within 2e-3 of that at 64 cells per wavelength, and the error falls as
    the square of the resolution (ratio 4 from 32 to 64 cells)."""
    fails = []
    for tau in (0.7, 1.3):
        r64, t64 = _decay_rate(lib, 64, tau)
        r32, t32 = _decay_rate(lib, 32, tau)
        e64, e32 = abs(r64 / t64 - 1), abs(r32 / t32 - 1)
        if not e64 < 2e-3:
            fails.append(f"shear decay tau={tau}: rel err {e64:.2e}")
        if not 3.5 < e32 / max(e64, 1e-300) < 4.5:
            fails.append(f"shear decay tau={tau}: not 2nd order ({e32:.2e} -> {e64:.2e})")
    return fails


def pin_taylor_green_decay(lib):
    """Force-free Taylor-Green vortex u = u0 (sin kx cos ky, -cos kx sin ky)
    decays as exp(-2 nu k^2 t), nu = (tau - 1/2)/3."""
    n = 48
    rho, ux, uy, k = inputs.taylor_green(n, n, u0=1e-4, rho0=0.2)
    lat = _lattice(lib, n, n, 1.5)
    lat.init_density(rho, ux, uy)
    tau = 0.9
    amps = []
    for _ in range(2):
        lat.step(150, oracle.NOFORCE, tau)
        _, vx, _ = lat.observe(noforce=True)
        amps.append(np.sum(vx * ux) / np.sum(ux * ux))
    rate = -np.log(amps[1] / amps[0]) / 150
    want = 2 * (tau - 0.5) / 3.0 * k ** 2
    return [] if abs(rate / want - 1) < 3e-3 else [f"TG rate {rate} want {want}"]


# ---------------------------------------------------------------------------
# the paper's physics: flat interface vs the mechanical-stability solution
# ---------------------------------------------------------------------------

def flat_interface(lib, t, scheme, tau, sigma, ny=100, nx=4, steps=30000,
                   tc_mode=0):
    """Coexistence densities of the Eq. 36 slab after relaxation (rho_g from
    the vapour rows 0 and ny-1, rho_l from the two central rows)."""
    T = th.temperature(t, tc_mode)
    rg, rl, _ = th.maxwell(th.CarnahanStarling(T))
    lat = oracle.Lattice(nx, ny, t, tc_mode=tc_mode, lib=lib)
    lat.init_density(inputs.slab_tanh(nx, ny, rg, rl, W=5.0))
    rc, _ = lat.step(steps, scheme, tau, sigma)
    if rc:
        return None
    rho, _, _ = lat.observe()
    return 0.5 * (rho[0].mean() + rho[-1].mean()), \
        0.5 * (rho[ny // 2 - 1].mean() + rho[ny // 2].mean())


def pin_improved_flat_interface(lib, temps=(0.8, 0.9), steps=30000):
    """Sec. IV B, Fig. 5: with the improved scheme the flat-interface
    coexistence densities follow the mechanical-stability solution (Eq. 26)
    at eps = 16 sigma (eps = -2(alpha + 24 G sigma)/beta, alpha = 0, beta = 3,
    G = -1): sigma = 0.0625 -> eps = 1, 0.125 -> eps = 2.  The theory keeps
    terms to second order only and the paper compares the two only by eye,
    read here as rho_l within 0.1 % and rho_g within 2 % (measured: 1e-4 and
    1.1 %)."""
    fails = []
    for t in temps:
        eos = th.CarnahanStarling(th.temperature(t))
        for sigma in (0.0625, 0.125):
            got = flat_interface(lib, t, oracle.IMPROVED, 0.8, sigma, steps=steps)
            want = th.mechanical_stability(eos, th.eps_of_sigma(sigma))
            if got is None:
                fails.append(f"T={t} sigma={sigma} diverged")
                continue
            if not (abs(got[1] / want[1] - 1) < 1e-3 and abs(got[0] / want[0] - 1) < 2e-2):
                fails.append(f"T={t} sigma={sigma}: sim {got} theory {want[:2]}")
    return fails


def pin_guo_flat_interface_is_eps0(lib):
    """Sec. IV A (text after Eq. 26 and Eq. 28): Guo's scheme adds no term to the
    macroscopic equations, so with nearest-neighbour interactions the flat
    interface obeys the mechanical-stability condition with eps = 0 (Eq. 6).
    The improved scheme with sigma = 0 is Guo's scheme (text after Eq. 31).
    A 2 x 100 slab relaxed for 2e4 steps reproduces the Eq. 6 solution at
    T/Tc = 0.85 to 1e-5 in rho_g and 1e-7 in rho_l."""
    t = 0.85
    want = th.mechanical_stability(th.CarnahanStarling(th.temperature(t)), 0.0)
    got = flat_interface(lib, t, oracle.IMPROVED, 1.0, 0.0, ny=100, nx=2, steps=20000)
    if got is None:
        return ["Guo slab diverged"]
    fails = _close("Guo rho_g vs eps=0", got[0], want[0], rtol=1e-5)
    fails += _close("Guo rho_l vs eps=0", got[1], want[1], rtol=1e-7)
    return fails


def pin_static_interface_actual_velocity(lib):
    """Table I: the actual fluid velocity is v = u + F/(2 rho) for every scheme.
    A relaxed static slab carries no mass flux, so v vanishes (to rounding)
    while u = -F/(2 rho) does not."""
    fails = []
    t = 0.9
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(t)))
    for sch, sig in ((oracle.SC, 0.0), (oracle.EDM, 0.0), (oracle.IMPROVED, 0.1)):
        lat = oracle.Lattice(2, 40, t, lib=lib)
        lat.init_density(inputs.slab_tanh(2, 40, rg, rl, W=5.0))
        if lat.step(8000, sch, 0.8, sig)[0]:
            fails.append(f"slab s={sch} diverged")
            continue
        _, vx, vy = lat.observe()
        _, ux, uy = oracle.moments(lat.f, lib=lib)
        if not (np.abs(vy).max() < 1e-12 and np.abs(vx).max() < 1e-12
                and np.abs(uy).max() > 1e-2):
            fails.append(f"s={sch}: max|v| {np.abs(vy).max():.2e} max|u| {np.abs(uy).max():.2e}")
    return fails


def pin_init_at_rest(lib):
    """A density field at rest (zero actual velocity v = u + F/(2 rho),
    Table I): for a uniform density it is the plain equilibrium at u = 0
    (F = 0 there); for the density of a slab the dynamics have relaxed to a
    static state, its velocity must be the relaxed state's own u (which the
    step computed, not the initialisation), and it is not zero."""
    fails = []
    t = 0.9
    uni = np.full((5, 4), 0.2)
    a = oracle.Lattice(4, 5, t, lib=lib)
    a.init_density_at_rest(uni)
    fails += _close("uniform at rest", a.f, oracle.init_equilibrium(uni, lib=lib))
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(t)))
    lat = oracle.Lattice(2, 40, t, lib=lib)
    lat.init_density(inputs.slab_tanh(2, 40, rg, rl, W=5.0))
    if lat.step(8000, oracle.SC, 0.8, 0.0)[0]:
        return fails + ["relaxing slab diverged"]
    rho_r, ux_r, uy_r = oracle.moments(lat.f, lib=lib)
    b = oracle.Lattice(2, 40, t, lib=lib)
    b.init_density_at_rest(rho_r)
    rho_b, ux_b, uy_b = oracle.moments(b.f, lib=lib)
    fails += _close("at-rest density", rho_b, rho_r, rtol=1e-14)
    fails += _close("at-rest u_y vs relaxed", uy_b, uy_r, atol=1e-11)
    fails += _close("at-rest u_x vs relaxed", ux_b, ux_r, atol=1e-11)
    if not np.abs(uy_r).max() > 1e-2:
        fails.append(f"relaxed slab has no u: {np.abs(uy_r).max():.2e}")
    return fails


# ---------------------------------------------------------------------------
# multiple-relaxation-time form of the improved scheme (end of Sec. IV)
# ---------------------------------------------------------------------------

def _mrt_basis():
    """D2Q9 moment basis (Lallemand-Luo): density, energy, energy square,
    momentum x, energy flux x, momentum y, energy flux y, two stresses."""
    ex, ey = EX.astype(float), EY.astype(float)
    c2 = ex ** 2 + ey ** 2
    return np.array([np.ones(Q), -4 + 3 * c2, 4 - 10.5 * c2 + 4.5 * c2 ** 2, ex,
                     (-5 + 3 * c2) * ex, ey, (-5 + 3 * c2) * ey, ex ** 2 - ey ** 2, ex * ey])


def pin_mrt_reduces_to_improved(lib):
    """With every rate 1/tau the MRT form must be Eq. 31 itself."""
    fails = []
    rng = np.random.default_rng(31)
    lib.oracle_set_mrt_rates(0.0, 0.0, 0.0)
    for _ in range(10):
        f = _random_cell(rng)
        Fx, Fy = rng.uniform(-2e-3, 2e-3, 2)
        psi = rng.uniform(0.1, 0.5)
        for tau in (0.6, 1.3):
            a = oracle.collide_cell(oracle.MRT, tau, 0.1, f, Fx, Fy, psi, lib=lib)
            b = oracle.collide_cell(oracle.IMPROVED, tau, 0.1, f, Fx, Fy, psi, lib=lib)
            fails += _close("MRT at rates 1/tau vs Eq. 31", a, b, rtol=1e-13, atol=1e-17)
    return fails


def pin_mrt_moment_relaxation(lib):
    """Post-collision moments against the closed-form D2Q9 moments of
    f_eq(rho, v) and of the improved forcing term: m* = m - s (m - m_eq) +
    (1 - s/2) S with m_eq = (rho, -2rho + 3rho|v|^2, rho - 3rho|v|^2, rho v_x,
    -rho v_x, rho v_y, -rho v_y, rho (v_x^2 - v_y^2), rho v_x v_y) and S = (0,
    6 v'.F, -6 v'.F, F_x, -F_x, F_y, -F_y, 2 (v'_x F_x - v'_y F_y),
    v'_x F_y + v'_y F_x)."""
    fails = []
    M = _mrt_basis()
    rng = np.random.default_rng(32)
    se, seps, sq, tau, sigma = 0.8, 1.1, 1.3, 0.7, 0.1
    lib.oracle_set_mrt_rates(se, seps, sq)
    try:
        for _ in range(10):
            f = _random_cell(rng)
            Fx, Fy = rng.uniform(-2e-3, 2e-3, 2)
            psi = rng.uniform(0.1, 0.5)
            out = oracle.collide_cell(oracle.MRT, tau, sigma, f, Fx, Fy, psi, lib=lib)
            m, mo = M @ f, M @ out
            rho = m[0]
            vx, vy = m[3] / rho + Fx / (2 * rho), m[5] / rho + Fy / (2 * rho)
            vpx = vx + sigma * Fx / ((tau - 0.5) * psi ** 2)
            vpy = vy + sigma * Fy / ((tau - 0.5) * psi ** 2)
            v2 = vx * vx + vy * vy
            meq = np.array([rho, -2 * rho + 3 * rho * v2, rho - 3 * rho * v2, rho * vx,
                            -rho * vx, rho * vy, -rho * vy, rho * (vx * vx - vy * vy),
                            rho * vx * vy])
            vF = vpx * Fx + vpy * Fy
            S = np.array([0.0, 6 * vF, -6 * vF, Fx, -Fx, Fy, -Fy, 2 * (vpx * Fx - vpy * Fy),
                          vpx * Fy + vpy * Fx])
            rate = np.array([1 / tau, se, seps, 1 / tau, sq, 1 / tau, sq, 1 / tau, 1 / tau])
            fails += _close("MRT moments", mo, m - rate * (m - meq) + (1 - rate / 2) * S,
                            atol=4e-15)
    finally:
        lib.oracle_set_mrt_rates(0.0, 0.0, 0.0)
    return fails


ALL_FAST_PINS = [
    pin_feq_moments, pin_force_stencil_taylor, pin_force_pair_antisymmetry,
    pin_stream_moves_along_e, pin_table1_forcing_moments, pin_paper_rewrites,
    pin_collision_momentum, pin_eos_and_psi, pin_step_conservation,
    pin_uniform_fixed_point, pin_shear_wave_decay, pin_taylor_green_decay,
    pin_guo_flat_interface_is_eps0, pin_static_interface_actual_velocity,
    pin_init_at_rest, pin_mrt_reduces_to_improved, pin_mrt_moment_relaxation,
]
