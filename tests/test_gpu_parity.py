"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: FP64 storage agrees to rounding (1e-13 per step, 1e-11
after 1e4 steps); FP32 to 1e-4 relative density after 1e4 steps (and 2e-6 of
the population scale per step); 16-bit deviation storage is reported and
gated loosely."""
import ctypes
import gc

import numpy as np
import pytest

import oracle
from oracle import theory as th
from paper_1204_4098_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

SCHEMES = [(lbm.SC, 0.0), (lbm.EDM, 0.0), (lbm.IMPROVED, 0.1), (lbm.NOFORCE, 0.0),
           (lbm.EDM_MOD, 0.0), (lbm.LADD, 0.0)]


def maxwell(t, tc_mode=0):
    return th.maxwell(th.CarnahanStarling(th.temperature(t, tc_mode)))[:2]


def droplet_state(nx, ny, t=0.9, seed=5):
    rg, rl = maxwell(t)
    rho = inputs.droplet(nx, ny, rg, rl, min(nx, ny) / 4.0, W=4.0)
    rng = np.random.default_rng(seed)
    ux = 0.01 * rng.uniform(-1, 1, (ny, nx))
    uy = 0.01 * rng.uniform(-1, 1, (ny, nx))
    return rho, ux, uy


def run_pair(nx, ny, t, rho, ux, uy, scheme, tau, sigma, steps, precision):
    gpu = lbm.Lattice(nx, ny, t, precision=precision)
    gpu.init_density(rho, ux, uy)
    gpu.step(steps, scheme, tau, sigma)
    ref = oracle.Lattice(nx, ny, t)
    ref.init_density(rho, ux, uy)
    rc, _ = ref.step(steps, scheme, tau, sigma)
    assert rc == 0
    return gpu, ref


@pytest.mark.parametrize("scheme,sigma", SCHEMES)
@pytest.mark.parametrize("steps", [1, 20])
def test_populations_fp32(scheme, sigma, steps):
    nx, ny, t = 45, 37, 0.9  # two strips (one ragged), rows not a band multiple
    rho, ux, uy = droplet_state(nx, ny, t)
    gpu, ref = run_pair(nx, ny, t, rho, ux, uy, scheme, 0.8, sigma, steps, lbm.FP32)
    fg, fo = gpu.populations(), ref.f
    err = np.max(np.abs(fg - fo)) / np.max(np.abs(fo))
    assert err < 2e-6 * steps ** 0.5, err
    rg, vxg, vyg = gpu.observe()
    ro, vxo, vyo = ref.observe()
    assert np.max(np.abs(rg / ro - 1)) < 2e-6 * steps ** 0.5
    assert np.max(np.abs(vxg - vxo)) < 1e-6 and np.max(np.abs(vyg - vyo)) < 1e-6


@pytest.mark.parametrize("scheme,sigma", SCHEMES)
@pytest.mark.parametrize("precision,tol", [(lbm.FP32, 2e-6), (lbm.FP64, 1e-13)])
def test_pair_kernel_populations_against_oracle(scheme, sigma, precision, tol):
    """The two-columns-per-lane kernel (the bench's kernel) against the oracle
    directly: 200 x 67 is three full 64-column strips and a ragged one."""
    nx, ny, t, steps = 200, 67, 0.9, 20
    rho, ux, uy = droplet_state(nx, ny, t)
    gpu = lbm.Lattice(nx, ny, t, precision=precision)
    gpu.set_variant(lbm.VARIANT_PAIR)
    assert gpu.variant() == lbm.VARIANT_PAIR
    gpu.init_density(rho, ux, uy)
    gpu.step(steps, scheme, 0.8, sigma)
    ref = oracle.Lattice(nx, ny, t)
    ref.init_density(rho, ux, uy)
    assert ref.step(steps, scheme, 0.8, sigma)[0] == 0
    err = np.max(np.abs(gpu.populations() - ref.f)) / np.max(np.abs(ref.f))
    assert err < tol * steps ** 0.5, err


@pytest.mark.parametrize("scheme,sigma", SCHEMES)
def test_populations_fp64(scheme, sigma):
    nx, ny, t = 45, 37, 0.9
    rho, ux, uy = droplet_state(nx, ny, t)
    for steps in (1, 25):
        gpu, ref = run_pair(nx, ny, t, rho, ux, uy, scheme, 0.8, sigma, steps, lbm.FP64)
        fg, fo = gpu.populations(), ref.f
        assert np.max(np.abs(fg - fo)) / np.max(np.abs(fo)) < 1e-13
        rg, vxg, vyg = gpu.observe()
        ro, vxo, vyo = ref.observe()
        assert np.max(np.abs(rg - ro)) < 1e-14
        assert np.max(np.abs(vxg - vxo)) < 1e-13 and np.max(np.abs(vyg - vyo)) < 1e-13


@pytest.mark.parametrize("nx,ny", [(1, 5), (5, 1), (1, 1), (3, 3), (5, 4), (31, 2), (32, 32),
                                   (33, 65), (64, 3), (97, 9)])
def test_edge_sizes_fp64(nx, ny):
    t = 0.9
    rg, rl = maxwell(t)
    rho = rg + (rl - rg) * np.random.default_rng(nx * 100 + ny).uniform(0.3, 0.7, (ny, nx))
    gpu, ref = run_pair(nx, ny, t, rho, None, None, lbm.IMPROVED, 0.9, 0.1, 5, lbm.FP64)
    assert np.max(np.abs(gpu.populations() - ref.f)) < 1e-13


# --- config 1: 64 x 64 flat interface, Shan-Chen, tau = 1, T = 0.8 Tc, 1e4 steps ---

_CONFIG1 = {}


def config1_oracle():
    if "ref" not in _CONFIG1:
        nx = ny = 64
        rg, rl = maxwell(0.8)
        rho0 = inputs.slab_step(nx, ny, rg, rl, 16, 48, amp=1e-3, seed=1)
        ref = oracle.Lattice(nx, ny, 0.8)
        ref.init_density(rho0)
        rc, _ = ref.step(10000, oracle.SC, 1.0)
        assert rc == 0
        _CONFIG1.update(rho0=rho0, ref=ref.observe(), mass0=float(rho0.sum()))
    return _CONFIG1


@pytest.mark.parametrize("precision,tol", [(lbm.FP32, 1e-4), (lbm.FP64, 1e-11)])
def test_config1_flat_interface_1e4_steps(precision, tol):
    c = config1_oracle()
    gpu = lbm.Lattice(64, 64, 0.8, precision=precision)
    gpu.init_density(c["rho0"])
    gpu.step(10000, lbm.SC, 1.0)
    rho, vx, vy = gpu.observe()
    err = np.max(np.abs(rho / c["ref"][0] - 1))
    assert err <= tol, err
    # coexistence densities (vapour rows 0, ny-1; liquid rows ny/2-1, ny/2)
    rg = 0.5 * (rho[0].mean() + rho[-1].mean())
    rl = 0.5 * (rho[31].mean() + rho[32].mean())
    mg, ml = maxwell(0.8)
    assert rl == pytest.approx(ml, rel=0.02) and 0.5 * mg < rg < 2 * mg


_CONFIG1_SCHEMES = {}


def config1_oracle_scheme(scheme, tau, sigma):
    """Config 1's slab (64 x 64, T = 0.8 Tc, Maxwell densities, noise 1e-3
    seed 1) after 2000 and after 1e4 steps of the given scheme in the FP64
    oracle (its OpenMP build, bit-identical to the plain one, when gcc has
    OpenMP)."""
    key = (scheme, tau, sigma)
    if key not in _CONFIG1_SCHEMES:
        rg, rl = maxwell(0.8)
        rho0 = inputs.slab_step(64, 64, rg, rl, 16, 48, amp=1e-3, seed=1)
        lib, _ = oracle.load_omp()
        ref = oracle.Lattice(64, 64, 0.8, lib=lib)
        ref.init_density(rho0)
        assert ref.step(2000, scheme, tau, sigma)[0] == 0
        early = ref.observe()
        assert ref.step(8000, scheme, tau, sigma)[0] == 0
        _CONFIG1_SCHEMES[key] = (rho0, early, ref.observe())
    return _CONFIG1_SCHEMES[key]


def interface_width(rho):
    """(rho_l - rho_g) / max_y |d rho/dy| of the row means, central differences
    (the width of an exact Eq. 36 tanh profile).  Sampled near the
    inflection point, it moves only by ~|shift| |d3 rho/dy3| / (2 max |d rho/dy|)
    under a sub-cell translation of the interface (< 5e-4 relative for a
    shift below 2e-3 cells on this slab)."""
    prof = rho.mean(1)
    grad = 0.5 * (np.roll(prof, -1) - np.roll(prof, 1))
    return (prof.max() - prof.min()) / np.abs(grad).max()


@pytest.mark.parametrize("variant", [lbm.VARIANT_PAIR, lbm.VARIANT_REGISTER])
@pytest.mark.parametrize("scheme,tau,sigma", [(lbm.SC, 1.0, 0.0), (lbm.EDM, 1.0, 0.0),
                                              (lbm.IMPROVED, 1.0, 0.1), (lbm.EDM, 0.8, 0.0),
                                              (lbm.IMPROVED, 0.8, 0.1)])
@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64])
def test_config1_1e4_steps_each_scheme_and_kernel(variant, scheme, tau, sigma, precision):
    """Config 1 (64 x 64 slab, 1e4 steps) against the FP64 oracle with the
    kernel variant forced: PAIR (two columns per lane, the bench's kernel)
    and REGISTER (one column per lane), for Shan-Chen (Eqs. 9-10), EDM
    (Eq. 11) and the improved scheme (Eq. 31, sigma = 0.1), at config 1's
    tau = 1 and at tau = 0.8 (where EDM and Shan-Chen differ).

    FP64: element-wise, relative density and velocity error 1e-11 after 2000
    and 1e4 steps.  FP32: element-wise 1e-4 after 2000 steps.  After 1e4
    steps the FP32 slab's two interfaces have each wandered by up to ~1e-3
    cells: FP32 rounding of the populations gives the total momentum a random
    walk (~1e-5), and an interface of a periodic slab is a nearly neutral
    mode (moving it only changes the bulk densities through the fixed mass).
    The element-wise error is then that shift times the interface gradient
    (2e-4 to 5e-4 measured, different for every rounding realisation,
    IEEE divisions included), so the FP32 gate there is on what does not
    depend on it: the coexistence densities (row-mean extremes) 1e-5, the
    field's variation along x 1e-5 of the largest density, each interface's
    shift below 2e-3 cells, and the interface width 1e-3."""
    rho0, early, (ro, vxo, vyo) = config1_oracle_scheme(scheme, tau, sigma)
    gpu = lbm.Lattice(64, 64, 0.8, precision=precision)
    gpu.set_variant(variant)
    assert gpu.variant() == variant
    gpu.init_density(rho0)
    tol = 1e-4 if precision == lbm.FP32 else 1e-11
    # after 2000 steps: element-wise for both precisions
    gpu.step(2000, scheme, tau, sigma)
    rho, vx, vy = gpu.observe()
    assert np.max(np.abs(rho / early[0] - 1)) <= tol
    verr = max(np.max(np.abs(vx - early[1])), np.max(np.abs(vy - early[2]))) / np.max(early[0])
    assert verr <= tol, verr
    gpu.step(8000, scheme, tau, sigma)
    rho, vx, vy = gpu.observe()
    if precision == lbm.FP64:
        assert np.max(np.abs(rho / ro - 1)) <= tol
        verr = max(np.max(np.abs(vx - vxo)), np.max(np.abs(vy - vyo))) / np.max(ro)
        assert verr <= tol, verr
        return
    coex = lambda r: np.array([r.mean(1).min(), r.mean(1).max()])
    assert np.max(np.abs(coex(rho) / coex(ro) - 1)) <= 1e-5
    xvar = np.max(np.abs((rho - rho.mean(1, keepdims=True)) - (ro - ro.mean(1, keepdims=True))))
    assert xvar <= 1e-5 * np.max(ro), xvar
    shift = interface_positions(rho) - interface_positions(ro)
    assert np.max(np.abs(shift)) < 2e-3, shift
    assert abs(interface_width(rho) / interface_width(ro) - 1) <= 1e-3


def interface_positions(rho):
    """Sub-cell y positions where the row-mean profile crosses its mid value."""
    prof = rho.mean(1)
    mid = 0.5 * (prof.max() + prof.min())
    out = []
    for y in range(len(prof) - 1):
        if (prof[y] - mid) * (prof[y + 1] - mid) < 0:
            out.append(y + (mid - prof[y]) / (prof[y + 1] - prof[y]))
    return np.array(out)


@pytest.mark.parametrize("precision,coex_tol,max_shift",
                         [(lbm.FP16DEV, 1e-3, 0.25), (lbm.BF16DEV, 5e-3, None)])
def test_config1_16bit_deviation_storage(precision, coex_tol, max_shift):
    """Deviation storage d_a = f_a - w_a rho in 16 bits with FP32 arithmetic.
    The density plane absorbs the rounding of the deviations, so mass is
    conserved; momentum is not.  The periodic slab's translation is undamped,
    so rounding noise makes it random-walk (fp16: a few hundredths of a cell
    in 1e4 steps; bf16, 8-bit mantissa: up to several cells), which the
    pointwise error at the steep interface magnifies.  Gated: the
    translation-invariant coexistence densities (minimum and maximum of the
    row means), mass, and for fp16 the interface shift; the pointwise error
    is printed."""
    c = config1_oracle()
    gpu = lbm.Lattice(64, 64, 0.8, precision=precision)
    gpu.init_density(c["rho0"])
    m0 = gpu.mass()
    gpu.step(10000, lbm.SC, 1.0)
    rho, _, _ = gpu.observe()
    ref = c["ref"][0]
    coex = lambda r: np.array([r.mean(1).min(), r.mean(1).max()])
    coex_err = np.max(np.abs(coex(rho) / coex(ref) - 1))
    shift = np.max(np.abs(interface_positions(rho) - interface_positions(ref)))
    point = np.max(np.abs(rho / ref - 1))
    print(f"16-bit storage {precision}: coexistence rel err {coex_err:.2e}, interface shift "
          f"{shift:.3f} cells, pointwise max rel err {point:.2e}, mass drift "
          f"{abs(gpu.mass() / m0 - 1):.1e}")
    assert coex_err < coex_tol
    if max_shift is not None:
        assert shift < max_shift
    assert abs(gpu.mass() / m0 - 1) < 2e-5  # FP32 rounding of the density plane


@pytest.mark.parametrize("precision,tol", [(lbm.FP64, 1e-13), (lbm.FP32, 1e-6)])
def test_mass_conservation(precision, tol):
    nx, ny, t = 70, 50, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    gpu = lbm.Lattice(nx, ny, t, precision=precision)
    gpu.init_density(rho, ux, uy)
    m0 = gpu.mass()
    assert m0 == pytest.approx(rho.sum(), rel=1e-7 if precision == lbm.FP32 else 1e-14)
    gpu.step(1000, lbm.IMPROVED, 0.7, 0.105)
    assert abs(gpu.mass() / m0 - 1) < tol


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64, lbm.BF16DEV])
def test_band_rows_do_not_change_results(precision):
    """The psi halo computed by a neighbouring warp equals the value the owning
    lane computes, so the result is bit-identical for any band height."""
    nx, ny, t = 77, 53, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    out = []
    for rows in (0, 1, 2, 5, 16, 53):
        gpu = lbm.Lattice(nx, ny, t, precision=precision)
        gpu.set_band_rows(rows)
        gpu.init_density(rho, ux, uy)
        gpu.step(30, lbm.IMPROVED, 0.8, 0.1)
        out.append(gpu.populations())
    for f in out[1:]:
        assert np.array_equal(f, out[0])


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64, lbm.BF16DEV])
def test_step_graphs_match_single_launches(precision):
    """Runs of 16 steps or more on a small lattice replay a captured graph of
    16 steps; the result equals one launch per step, from either buffer
    parity, with a remainder, and after the scheme, tau, the band height or
    the kernel variant changed (each change captures a new graph)."""
    nx, ny, t = 66, 40, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    runs = [(37, lbm.IMPROVED, 0.8, 0.1, 0, lbm.VARIANT_AUTO),
            (4, lbm.IMPROVED, 0.8, 0.1, 0, lbm.VARIANT_AUTO),
            (32, lbm.IMPROVED, 0.8, 0.1, 0, lbm.VARIANT_AUTO),
            (16, lbm.IMPROVED, 0.9, 0.1, 0, lbm.VARIANT_AUTO),
            (17, lbm.EDM, 0.9, 0.0, 0, lbm.VARIANT_AUTO),
            (16, lbm.EDM, 0.9, 0.0, 3, lbm.VARIANT_AUTO),
            (16, lbm.EDM, 0.9, 0.0, 3, lbm.VARIANT_REGISTER),
            (48, lbm.IMPROVED, 0.8, 0.1, 0, lbm.VARIANT_AUTO)]
    graph = lbm.Lattice(nx, ny, t, precision=precision)
    single = lbm.Lattice(nx, ny, t, precision=precision)
    for g in (graph, single):
        g.init_density(rho, ux, uy)
    for n, scheme, tau, sigma, rows, variant in runs:
        for g in (graph, single):
            g.set_band_rows(rows)
            g.set_variant(variant)
        graph.step(n, scheme, tau, sigma)
        for _ in range(n):
            single.step(1, scheme, tau, sigma)
        assert np.array_equal(graph.populations(), single.populations()), (n, scheme, tau)
    graph.close()
    single.close()


def test_step_graphs_of_the_staged_kernel_match_single_launches():
    """The same for the bulk-copy staged kernel (its tensor maps are kernel
    arguments captured with the graph)."""
    nx, ny, t = 64, 40, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    out = []
    for chunk in (40, 1):
        g = lbm.Lattice(nx, ny, t, precision=lbm.FP32)
        g.set_variant(lbm.VARIANT_STAGED)
        g.init_density(rho, ux, uy)
        for _ in range(40 // chunk):
            g.step(chunk, lbm.IMPROVED, 0.8, 0.1)
        out.append(g.populations())
        g.close()
    assert np.array_equal(out[0], out[1])


def test_moments_of_a_lattice_with_fewer_rows_than_chunks():
    """A 1,398,102 x 3 lattice (4.19 M cells: chunked moments, one chunk
    empty) observed against the oracle on the same populations."""
    nx, ny, t = 1398102, 3, 0.85
    rg, rl = maxwell(t)
    rng = np.random.default_rng(11)
    rho = 0.5 * (rg + rl) * (1.0 + 0.01 * rng.uniform(-1, 1, (ny, nx)))
    gpu = lbm.Lattice(nx, ny, t, precision=lbm.FP32)
    gpu.init_density(rho)
    gpu.step(2, lbm.IMPROVED, 0.8, 0.1)
    ref = oracle.Lattice(nx, ny, t)
    ref.f = gpu.populations()
    ref.last_scheme = oracle.IMPROVED
    want = ref.observe()
    got = gpu.observe()
    assert np.max(np.abs(got[0] - want[0]) / want[0]) < 2e-6
    for k in (1, 2):
        assert np.max(np.abs(got[k] - want[k])) < 2e-5, k
    gpu.close()


def test_steps_captured_into_a_caller_graph_replay_exactly():
    """lbm_step_async on a stream the caller is capturing records one launch
    per step into the caller's graph (no graph of its own); two replays of 32
    captured steps equal 64 steps run directly."""
    torch = pytest.importorskip("torch")
    nx, ny, t = 66, 40, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    s = torch.cuda.Stream()
    a = lbm.Lattice(nx, ny, t, stream=s.cuda_stream)
    b = lbm.Lattice(nx, ny, t)
    a.init_density(rho, ux, uy)
    b.init_density(rho, ux, uy)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        a.step_async(32, lbm.IMPROVED, 0.8, 0.1)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    b.step(64, lbm.IMPROVED, 0.8, 0.1)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


@pytest.mark.parametrize("precision,rtol,vtol", [(lbm.FP64, 1e-11, 1e-12),
                                                 (lbm.FP32, 2e-6, 2e-5)])
def test_moments_of_a_large_lattice_in_row_chunks(precision, rtol, vtol):
    """From 2048^2 cells on, lbm_get_moments computes and copies the rows in
    chunks (each chunk copied while the next is computed).  Every row, the
    chunk boundaries included, equals the oracle's observation (Table I:
    v = u + F / (2 rho)) of the same populations; pinned and pageable
    outputs agree bitwise."""
    torch = pytest.importorskip("torch")
    nx, ny, t = 2048, 2050, 0.85  # ny not a multiple of the chunk count
    rg, rl = maxwell(t)
    rho = inputs.droplet(nx, ny, rg, rl, 300.0, W=4.0)
    gpu = lbm.Lattice(nx, ny, t, precision=precision)
    gpu.init_density(rho)
    gpu.step(3, lbm.IMPROVED, 0.8, 0.1)
    ref = oracle.Lattice(nx, ny, t)
    ref.f = gpu.populations()
    ref.last_scheme = oracle.IMPROVED
    want = ref.observe()
    pin = [torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy() for _ in range(3)]
    got = gpu.observe(out=tuple(pin))
    pageable = gpu.observe()
    for a, b in zip(got, pageable):
        assert np.array_equal(a, b)
    assert np.max(np.abs(got[0] - want[0]) / want[0]) < rtol
    for k in (1, 2):
        assert np.max(np.abs(got[k] - want[k])) < vtol, k
    # the outputs are written independently: rho alone equals rho of all three
    rho_only = np.empty((ny, nx))
    assert lbm.lib().lbm_get_moments(gpu.ctx, lbm._dptr(rho_only), None, None) == lbm.LBM_OK
    assert np.array_equal(rho_only, got[0])
    gpu.close()


def test_checkpoint_roundtrip_is_bitwise():
    nx, ny, t = 64, 40, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    for precision in (lbm.FP32, lbm.FP64):
        a = lbm.Lattice(nx, ny, t, precision=precision)
        a.init_density(rho, ux, uy)
        a.step(40, lbm.EDM, 0.7)
        b = lbm.Lattice(nx, ny, t, precision=precision)
        a.step(10, lbm.EDM, 0.7)
        b.set_populations(a.populations())
        a.step(10, lbm.EDM, 0.7)
        b.step(10, lbm.EDM, 0.7)
        assert np.array_equal(a.populations(), b.populations())


def test_noforce_taylor_green_fp32_vs_oracle():
    n = 48
    rho, ux, uy, k = inputs.taylor_green(n, n, u0=1e-3, rho0=0.2)
    gpu, ref = run_pair(n, n, 1.5, rho, ux, uy, lbm.NOFORCE, 0.9, 0.0, 300, lbm.FP32)
    _, vxg, vyg = gpu.observe()
    _, vxo, vyo = ref.observe()
    # FP32 populations resolve u to ~1e-8 per step; 300 steps random-walk to ~1e-7
    assert np.max(np.abs(vxg - vxo)) < 5e-7 and np.max(np.abs(vyg - vyo)) < 5e-7


def test_divergence_is_reported_and_context_survives():
    nx, ny, t = 40, 30, 0.8
    rg, rl = maxwell(t)
    rho = inputs.slab_step(nx, ny, rg, rl)
    f = oracle.init_equilibrium(rho)
    f[:, 10, 10] *= 1.2 / rho[10, 10]  # rho = 1.2 > 4/b: outside the domain of psi
    gpu = lbm.Lattice(nx, ny, t)
    gpu.set_populations(f)
    assert gpu.step(3, lbm.SC, 1.0, raise_on_error=False) == lbm.LBM_E_DIVERGED
    gpu.init_density(rho)
    assert gpu.step(3, lbm.SC, 1.0, raise_on_error=False) == lbm.LBM_OK


def test_invalid_arguments():
    gpu = lbm.Lattice(16, 16, 0.8)
    with pytest.raises(lbm.LbmError) as e:
        gpu.step(1, lbm.SC, 1.0)
    assert e.value.status == lbm.LBM_E_STATE
    bad = np.full((16, 16), 0.2)
    bad[3, 3] = 1.5
    with pytest.raises(lbm.LbmError) as e:
        gpu.init_density(bad)
    assert e.value.status == lbm.LBM_E_INVAL
    gpu.init_density(np.full((16, 16), 0.2))
    for args in ((1, lbm.SC, 0.5), (1, 17, 1.0), (-1, lbm.SC, 1.0), (1, lbm.SC, float("nan"))):
        assert gpu.step(*args, raise_on_error=False) == lbm.LBM_E_INVAL
    assert gpu.step(0, lbm.SC, 1.0, raise_on_error=False) == lbm.LBM_OK


# --- full size: 8192 x 8192 spinodal decomposition, improved scheme -------------

def _one_step_rho_at(rho0, RT, y, x, tau, sigma, scheme=oracle.IMPROVED):
    """rho(x, t=1) from f(., 0) = f_eq(rho0, 0), by the oracle's own primitives
    on the 5x5 neighbourhood (psi radius 2 -> F radius 1 -> pull)."""
    ny, nx = rho0.shape
    ys = [(y + d) % ny for d in range(-2, 3)]
    xs = [(x + d) % nx for d in range(-2, 3)]
    win = rho0[np.ix_(ys, xs)]
    psi = np.array([[oracle.psi(r, RT) for r in row] for row in win])
    Fx, Fy = oracle.force(psi)
    total = 0.0
    for a in range(9):
        sy, sx = 2 - oracle.EY[a], 2 - oracle.EX[a]  # source cell x - e_a in the window
        fs = oracle.feq(win[sy, sx], 0.0, 0.0)
        post = oracle.collide_cell(scheme, tau, sigma, fs, Fx[sy, sx], Fy[sy, sx],
                                   psi[sy, sx])
        total += post[a]
    return total


@pytest.mark.parametrize("precision,scheme,sigma,rel,mass_tol",
                         [(lbm.FP32, lbm.IMPROVED, 0.1, 2e-6, 1e-9),
                          (lbm.FP32, lbm.SC, 0.0, 2e-6, 1e-9),
                          (lbm.FP32, lbm.EDM, 0.0, 2e-6, 1e-9),
                          (lbm.FP32, lbm.MRT, 0.1, 2e-6, 1e-9),
                          (lbm.BF16DEV, lbm.IMPROVED, 0.1, 1e-4, 1e-7),
                          (lbm.FP16DEV, lbm.IMPROVED, 0.1, 2e-5, 1e-7)],
                         ids=["fp32-improved", "fp32-sc", "fp32-edm", "fp32-mrt",
                              "bf16dev-improved", "fp16dev-improved"])
def test_full_size_8192_sampled_against_oracle(precision, scheme, sigma, rel, mass_tol):
    """The bench's lattice and kernel (8192^2, two columns per lane, rows
    copied into shared memory): the density after one step at sampled cells
    -- corners, strip and band edges, random cells -- against the oracle's
    step on each cell's neighbourhood.  16-bit deviation storage starts
    exact (the deviations of f_eq at rest are 0) and rounds the post-step
    deviations (|d| ~ 1e-3 of rho here) to 8 / 11 significant bits, summed
    over nine source cells: well inside 1e-4 / 2e-5 of rho."""
    n, t, tau = 8192, 0.85, 0.8
    rates = (0.8, 1.1, 1.3)
    rg, rl = maxwell(t)
    rho0 = inputs.spinodal(n, n, 0.5 * (rg + rl), amp=0.01, seed=3)
    gpu = lbm.Lattice(n, n, t, precision=precision)
    assert gpu.variant() == lbm.VARIANT_PAIR
    gpu.set_mrt_rates(*rates)
    gpu.init_density(rho0)
    m0 = gpu.mass()
    gpu.step(1, scheme, tau, sigma)
    rho1, _, _ = gpu.observe()
    RT = th.temperature(t)
    rng = np.random.default_rng(8)
    cells = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (4095, 31), (17, 32), (100, 63),
             (101, 64), (431, 127), (432, 128)]
    cells += [tuple(v) for v in rng.integers(0, n, (150, 2))]
    oracle.set_mrt_rates(*rates)
    try:
        for y, x in cells:
            want = _one_step_rho_at(rho0, RT, y, x, tau, sigma, scheme)
            assert rho1[y, x] == pytest.approx(want, rel=rel), (y, x)
    finally:
        oracle.set_mrt_rates(0.0, 0.0, 0.0)
    gpu.step(9, scheme, tau, sigma)
    assert abs(gpu.mass() / m0 - 1) < mass_tol
    gpu.close()


@pytest.mark.parametrize("nx,ny", [(64, 40), (68, 37), (100, 33), (128, 65), (132, 8)])
@pytest.mark.parametrize("scheme,sigma", [(lbm.SC, 0.0), (lbm.IMPROVED, 0.1), (lbm.NOFORCE, 0.0)])
def test_staged_kernel_matches_register_kernel_bitwise(nx, ny, scheme, sigma):
    """The bulk-copy staged step (rows in shared memory, periodic edges from a
    second copy, ragged last strip) computes exactly what the register step
    does, for every band height."""
    t = 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    out = []
    for variant, rows in ((lbm.VARIANT_REGISTER, 0), (lbm.VARIANT_STAGED, 0),
                          (lbm.VARIANT_STAGED, 1), (lbm.VARIANT_STAGED, 7)):
        g = lbm.Lattice(nx, ny, t, precision=lbm.FP32)
        g.set_variant(variant)
        g.set_band_rows(rows)
        g.init_density(rho, ux, uy)
        g.step(25, scheme, 0.8, sigma)
        out.append(g.populations())
    for f in out[1:]:
        assert np.array_equal(f, out[0])


def test_staged_kernel_fp32_parity_with_oracle():
    nx, ny, t = 68, 37, 0.9
    rho, ux, uy = droplet_state(nx, ny, t)
    gpu = lbm.Lattice(nx, ny, t, precision=lbm.FP32)
    gpu.set_variant(lbm.VARIANT_STAGED)
    gpu.init_density(rho, ux, uy)
    gpu.step(20, lbm.IMPROVED, 0.8, 0.1)
    ref = oracle.Lattice(nx, ny, t)
    ref.init_density(rho, ux, uy)
    assert ref.step(20, oracle.IMPROVED, 0.8, 0.1)[0] == 0
    err = np.max(np.abs(gpu.populations() - ref.f)) / np.max(np.abs(ref.f))
    assert err < 2e-6 * 20 ** 0.5, err


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64, lbm.BF16DEV, lbm.FP16DEV])
@pytest.mark.parametrize("nx,ny", [(2, 9), (4, 4), (2, 1), (64, 1), (66, 2), (40, 21), (64, 33),
                                   (66, 40), (100, 17), (130, 65)])
def test_pair_kernel_matches_register_kernel_bitwise(precision, nx, ny):
    """Two columns per lane (vector loads, shuffled +-1 pulls, boundary and
    halo elements from extra lanes, wrapped lanes in ragged strips, rows
    copied into shared memory ahead of use, bands of one row) computes
    exactly what one column per lane does: steps of every scheme and the
    observed density and velocity, in every storage type (16-bit deviation
    storage included: deviations and density plane pairs)."""
    t = 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    for scheme, sigma in ((lbm.SC, 0.0), (lbm.IMPROVED, 0.1), (lbm.EDM, 0.0),
                          (lbm.NOFORCE, 0.0)):
        out = []
        for variant, rows in ((lbm.VARIANT_REGISTER, 0), (lbm.VARIANT_PAIR, 0),
                              (lbm.VARIANT_PAIR, 1), (lbm.VARIANT_PAIR, 3)):
            g = lbm.Lattice(nx, ny, t, precision=precision)
            g.set_variant(variant)
            g.set_band_rows(rows)
            g.init_density(rho, ux, uy)
            g.step(15, scheme, 0.8, sigma)
            out.append((g.populations(), *g.observe()))
        for o in out[1:]:
            for a, b in zip(o, out[0]):
                assert np.array_equal(a, b), (scheme, variant)


def test_auto_variant_choice():
    """AUTO: two columns per lane for even nx on lattices large enough to occupy
    the GPU with 64-column strips, one column per lane otherwise (odd nx, FP64,
    small lattices); an explicit variant is honoured where it applies."""
    def variant(nx, ny, precision=lbm.FP32, want=None):
        g = lbm.Lattice(nx, ny, 0.85, precision=precision)
        if want is not None:
            g.set_variant(want)
        v = g.variant()
        g.close()
        return v
    assert variant(1024, 1024) == lbm.VARIANT_PAIR
    assert variant(1024, 1024, lbm.BF16DEV) == lbm.VARIANT_PAIR
    assert variant(1025, 1024) == lbm.VARIANT_REGISTER
    assert variant(1024, 1024, lbm.FP64) == lbm.VARIANT_REGISTER
    assert variant(256, 256) == lbm.VARIANT_REGISTER
    assert variant(256, 256, want=lbm.VARIANT_PAIR) == lbm.VARIANT_PAIR
    assert variant(1024, 1024, want=lbm.VARIANT_STAGED) == lbm.VARIANT_STAGED
    assert variant(1026, 64, want=lbm.VARIANT_STAGED) == lbm.VARIANT_REGISTER  # nx % 4 != 0


def test_grid_barrier_reports_timeout_and_context_survives():
    """The batch engine's grid barrier, with one CTA that never arrives, gives
    up after its spin limit and reports LBM_E_TIMEOUT; the device stays usable."""
    assert lbm.selftest_grid_barrier_timeout(0) == lbm.LBM_E_TIMEOUT
    g = lbm.Lattice(32, 32, 0.85, precision=lbm.FP32)
    g.init_density(np.full((32, 32), 0.2))
    g.step(5, lbm.SC, 1.0)
    assert np.all(np.isfinite(g.observe()[0]))


def test_bounded_wait_reports_timeout_and_context_survives():
    """A device wait on an mbarrier nothing arrives on gives up after its poll
    limit and reports LBM_E_TIMEOUT (no fault, no hang); the device is usable
    afterwards."""
    assert lbm.selftest_wait_timeout(0, polls=1000) == lbm.LBM_E_TIMEOUT
    nx, ny, t = 40, 36, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    g = lbm.Lattice(nx, ny, t, precision=lbm.FP32)
    g.init_density(rho, ux, uy)
    g.step(10, lbm.IMPROVED, 0.8, 0.1)
    assert np.all(np.isfinite(g.observe()[0]))


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP64, lbm.BF16DEV])
def test_uniform_density_stays_uniform_at_rest(precision):
    """Degenerate case: at a uniform density every cell sees the same
    neighbours, so psi's stencil gives F = 0 exactly and opposite populations
    stay equal: for every scheme (odd and even widths, both kernel variants)
    the state stays uniform cell for cell, the velocity exactly zero, and the
    density at its value to rounding (the collision's (1 - omega) f + omega
    f_eq need not round back to f)."""
    tol = {lbm.FP32: 1e-6, lbm.FP64: 1e-14, lbm.BF16DEV: 1e-6}[precision]
    for nx in (64, 33):
        rho = np.full((24, nx), 0.2)
        for scheme, sigma in ((lbm.SC, 0.0), (lbm.EDM, 0.0), (lbm.IMPROVED, 0.1),
                              (lbm.EDM_MOD, 0.0), (lbm.LADD, 0.0)):
            g = lbm.Lattice(nx, 24, 0.85, precision=precision)
            g.init_density(rho)
            g.step(50, scheme, 0.7, sigma)
            f = g.populations()
            assert np.all(f == f[:, :1, :1]), (nx, scheme)
            r, vx, vy = g.observe()
            assert not np.any(vx) and not np.any(vy), (nx, scheme)
            assert np.max(np.abs(r / 0.2 - 1)) < tol, (nx, scheme)
            g.close()


def test_host_alloc_buffers_carry_the_same_values():
    """lbm_host_alloc / lbm_host_free: zeroed page-locked buffers (aligned to
    a huge page from one huge page up) that init and moments read and write
    with the same values as pageable arrays; the argument errors."""
    L = lbm.lib()
    p = ctypes.c_void_p()
    assert L.lbm_host_alloc(0, ctypes.byref(p)) == lbm.LBM_E_INVAL
    assert L.lbm_host_alloc(16, None) == lbm.LBM_E_INVAL
    assert L.lbm_host_free(None) == lbm.LBM_OK
    assert L.lbm_host_alloc(40, ctypes.byref(p)) == lbm.LBM_OK
    assert L.lbm_host_free(ctypes.c_void_p(p.value + 8)) == lbm.LBM_E_INVAL
    assert L.lbm_host_free(p) == lbm.LBM_OK
    assert L.lbm_host_free(p) == lbm.LBM_E_INVAL  # already freed
    hp = 2 << 20
    try:
        hp = int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
    except OSError:
        pass
    big = lbm.host_array((hp // 8 + 3,))
    assert big.ctypes.data % hp == 0 and not big[::4096].any() and big[-1] == 0.0
    addr = big.ctypes.data
    view = big[1:]
    del big
    gc.collect()
    assert view[-1] == 0.0  # a view keeps the buffer
    del view
    gc.collect()
    # collected: the binding returned it through lbm_host_free already
    assert L.lbm_host_free(ctypes.c_void_p(addr)) == lbm.LBM_E_INVAL
    nx, ny, t = 70, 50, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)
    h = [lbm.host_array((ny, nx)) for _ in range(6)]
    h[0][...] = rho
    h[1][...] = ux
    h[2][...] = uy
    a = lbm.Lattice(nx, ny, t)
    b = lbm.Lattice(nx, ny, t)
    a.init_density(h[0], h[1], h[2])
    b.init_density(rho, ux, uy)
    a.step(20, lbm.IMPROVED, 0.8, 0.1)
    b.step(20, lbm.IMPROVED, 0.8, 0.1)
    got = a.observe(out=tuple(h[3:]))
    for x, y in zip(got, b.observe()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_pinned_host_arrays_are_used_in_place():
    """Page-locked host arrays are read and written by the kernels directly
    (no staging copy); the results equal those through pageable arrays, also
    with some outputs NULL."""
    torch = pytest.importorskip("torch")
    nx, ny, t = 96, 40, 0.85
    rho, ux, uy = droplet_state(nx, ny, t)

    def pinned(a):
        p = torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy()
        p[...] = a
        return p

    outs = []
    for use_pinned in (False, True):
        g = lbm.Lattice(nx, ny, t, precision=lbm.FP32)
        if use_pinned:
            g.init_density(pinned(rho), pinned(ux), pinned(uy))
        else:
            g.init_density(rho, ux, uy)
        g.step(30, lbm.IMPROVED, 0.8, 0.1)
        o = tuple(pinned(np.zeros((ny, nx))) for _ in range(3)) if use_pinned else None
        outs.append((g.populations(), *g.observe(out=o)))
        if use_pinned:
            r = pinned(np.zeros((ny, nx)))
            assert lbm.lib().lbm_get_moments(g.ctx, lbm._dptr(r), None, None) == lbm.LBM_OK
            assert np.array_equal(r, outs[-1][1])
        g.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision,tol,vtol", [(lbm.FP64, 1e-13, 1e-14),
                                                (lbm.FP32, 2e-7, 1e-7)])
def test_init_density_at_rest_matches_oracle(precision, tol, vtol):
    """lbm_init_density_at_rest: f = f_eq(rho, u) with u = -F/(2 rho) from the
    Eq. 3 force of rho itself.  Populations against the oracle's
    oracle_init_at_rest element-wise; the actual velocity of Table I, as
    lbm_get_moments reports it, vanishes while u = -F/(2 rho) does not."""
    nx, ny, t = 45, 37, 0.9
    rho, _, _ = droplet_state(nx, ny, t)
    gpu = lbm.Lattice(nx, ny, t, precision=precision)
    gpu.init_density_at_rest(rho)
    ref = oracle.Lattice(nx, ny, t)
    ref.init_density_at_rest(rho)
    err = np.max(np.abs(gpu.populations() - ref.f)) / np.max(np.abs(ref.f))
    assert err < tol, err
    _, vx, vy = gpu.observe()
    assert max(np.abs(vx).max(), np.abs(vy).max()) < vtol
    _, ux, uy = oracle.moments(ref.f)
    assert max(np.abs(ux).max(), np.abs(uy).max()) > 1e-3


def test_init_density_at_rest_rejects_density_outside_psi_domain():
    rho = np.full((9, 8), 0.2)
    rho[3, 4] = 1.2  # b rho / 4 >= 1
    gpu = lbm.Lattice(8, 9, 0.9)
    with pytest.raises(lbm.LbmError) as e:
        gpu.init_density_at_rest(rho)
    assert e.value.status == lbm.LBM_E_INVAL


def test_batch_init_density_at_rest():
    """The batch engine's at-rest start: zero actual velocity from its moments,
    the same populations as a single lattice started at rest."""
    nx, ny, t = 64, 48, 0.85
    rho, _, _ = droplet_state(nx, ny, t)
    inst = [dict(nx=nx, ny=ny, T_over_Tc=t, tau=0.8, sigma=0.1, scheme=lbm.IMPROVED)]
    with lbm.Batch(inst, conv=lbm.CONV_NONE, max_steps=1000) as b:
        b.init_density_at_rest(0, rho)
        r, vx, vy = b.moments(0)
    assert max(np.abs(vx).max(), np.abs(vy).max()) < 1e-7
    single = lbm.Lattice(nx, ny, t)
    single.init_density_at_rest(rho)
    assert np.max(np.abs(single.observe()[0] - r)) < 1e-7
