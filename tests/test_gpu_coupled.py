"""GPU parity of the coupled two-species systems of Section 8 (complex
Ginzburg-Landau with D = 1 + i alpha, cubic Schrodinger): the complex line
kernels, through etd_create_coupled, against the FP64 oracle's 2p x 2p block
solves on the same seeded inputs.

Errors are measured on the complex field u = u_0 + i u_1 as a whole:
max|U_gpu - U_oracle| / max|U_oracle| over both species (one component can be
near zero while the field is not, e.g. the imaginary part of the Schrodinger
example right after t = 0).
Tolerances: FP64 <= 1e-12 relative per step, times the number of steps for runs;
FP32: fp32_step_bound(w) per step (tests/tolerances.py: the decay factor of
the complex line matrices, the 17-fold cancellation of R = 9T - 8S, unit
roundoff 2^-24)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2001_11220_gb300 import workloads as W  # noqa: E402
from tests.dense_reference import oracle_problem  # noqa: E402
from tests.tolerances import fp32_step_bound  # noqa: E402

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
TWO_PI2 = 2.0 * math.pi ** 2


def rel_err(a, ref):
    return float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300))


def gpu_run(w, U0, nsteps, precision="fp64"):
    from paper_2001_11220_gb300.api import EtdRdpIf
    ctx = EtdRdpIf.from_workload(w, precision)
    U = torch.tensor(U0, device="cuda", dtype=ctx.dtype)
    ctx.run(U, 0.0, nsteps)
    torch.cuda.synchronize()
    info = ctx.info()
    ctx.close()
    return U.double().cpu().numpy(), info


def ccase(name, n, bc, Dc, reaction, params, k=0.05, ic="normal", length=None):
    return W.Workload(name, n, bc, (1.0, 1.0), reaction, params, k, 1, length=length, ic=ic,
                      ic_args=((0.3, -0.2), 0.5) if ic == "normal" else (), Dc=Dc)


NLS_C = 1.0 - TWO_PI2
CASES = [
    # complex Ginzburg-Landau, D = 1 + 0.8 i, periodic, ragged line lengths (not multiples of 32)
    ccase("cgl_alpha_2d", (48, 37), W.PERIODIC, (1.0, -0.8, 0.8, 1.0), "cgl", (1.3,), k=0.05,
          length=(24.0, 18.5)),
    ccase("cgl_alpha_3d", (20, 18, 13), W.PERIODIC, (1.0, -0.8, 0.8, 1.0), "cgl", (1.3,), k=0.05,
          length=(10.0, 9.0, 6.5)),
    # Section 8's Schrodinger problem (position term, Neumann) and a cubic periodic one
    ccase("nls_neu_2d", (33, 29), W.NEUMANN, (0.0, -1.0, 1.0, 0.0), "nls", (0.0, NLS_C, NLS_C), k=0.002,
          ic="nls_exact"),
    ccase("nls_per_3d", (16, 12, 10), W.PERIODIC, (0.0, -1.0, 1.0, 0.0), "nls", (0.3, -1.0, 0.0), k=0.01),
    ccase("nls_mixed_3d", (11, 9, 7), (W.NEUMANN, W.DIRICHLET, W.NEUMANN), (0.0, -1.0, 1.0, 0.0), "nls",
          (0.0, NLS_C, NLS_C), k=0.002, ic="nls_exact"),
    # linear reaction, Dirichlet, general p + i q; lines shorter than a warp (p = 5 < 32)
    ccase("lin_dir_2d", (5, 41), W.DIRICHLET, (0.3, -0.5, 0.5, 0.3), "linear", (-0.4, 0.1), k=0.02),
    # long x lines: several nodes per lane (300 nodes: 10 per lane, 11 after rounding to odd)
    ccase("cgl_long_x", (300, 9), (W.PERIODIC, W.NEUMANN), (1.0, 0.5, -0.5, 1.0), "cgl", (0.7,), k=0.05,
          length=(150.0, 4.5)),
    # lines past the unrolled chunk bounds (1500 and 700 nodes: 47 and 23 per lane, runtime loops),
    # Neumann x, Dirichlet y
    ccase("nls_runtime_chunks", (1500, 700), (W.NEUMANN, W.DIRICHLET), (0.0, -1.0, 1.0, 0.0), "nls",
          (0.2, -1.0, 0.0), k=0.01, length=(30.0, 14.0)),
    # d = 1 (one fused sweep per step): a periodic line (Sherman-Morrison) and a Dirichlet one
    ccase("cgl_1d_per", (77,), (W.PERIODIC,), (1.0, -0.8, 0.8, 1.0), "cgl", (1.3,), k=0.05, length=(38.5,)),
    ccase("lin_1d_dir", (45,), (W.DIRICHLET,), (0.3, -0.5, 0.5, 0.3), "linear", (-0.4, 0.1), k=0.02),
    # the longest FP64 line the kernel's shared memory takes (3000 nodes: one line per block)
    ccase("nls_max_line", (3000, 3), (W.NEUMANN, W.NEUMANN), (0.0, -1.0, 1.0, 0.0), "nls", (0.2, -1.0, 0.0),
          k=0.01, length=(60.0, 1.0)),
]


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_coupled_steps_fp64_match_oracle(w):
    U0 = W.initial_state(w)
    for nsteps in (1, 4):
        got, info = gpu_run(w, U0, nsteps)
        ref = oracle.run(oracle_problem(w), U0, 0.0, nsteps)
        e = rel_err(got, ref)
        print(f"{w.name} fp64 {nsteps} steps: {e:.2e}")
        assert e <= nsteps * FP64_TOL, (w.name, nsteps, e)
        assert np.max(np.abs(ref - U0)) > 1e-4  # the steps moved the state
    assert info["staged"][:w.dim] == [6] * w.dim and info["launches_per_step"] == w.dim


@pytest.mark.parametrize("w", CASES[:5], ids=lambda w: w.name)
def test_coupled_steps_fp32_within_bound(w):
    U0 = W.initial_state(w)
    got, _ = gpu_run(w, U0, 3, "fp32")
    ref = oracle.run(oracle_problem(w), U0, 0.0, 3)
    e, bound = rel_err(got, ref), 3 * fp32_step_bound(w)
    print(f"{w.name} fp32 3 steps: {e:.2e} (bound {bound:.2e})")
    assert e <= bound, (w.name, e, bound)


def test_real_coupling_equals_uncoupled_kernels():
    """Dm = diag(1, 1) through the complex kernels and D = (1, 1) through the real
    kernels (CGL with alpha = 0, periodic: the circulant family) solve the same
    problem: FP64 agreement to rounding."""
    w = W.cgl_2d(p=64, steps=5).with_(length=(32.0, 32.0))
    U0 = W.initial_state(w.with_(ic="normal", ic_args=((0.0, 0.0), 0.5)))
    a, _ = gpu_run(w, U0, 5)
    b, info = gpu_run(w.with_(Dc=(1.0, 0.0, 0.0, 1.0)), U0, 5)
    assert info["staged"][:2] == [6, 6]
    assert rel_err(b, a) <= 5 * FP64_TOL


def test_paper_schrodinger_2d_whole_run():
    """Section 8's 2D run: p = 79 (h = 1/78), k = 0.0125, T = 1 (80 steps): the GPU
    matches the oracle over the whole run.  At that k the scheme's error against
    the exact solution e^{-iT} cos(pi x) cos(pi y) is large (0.61 in the oracle:
    the potential q ~ 1 - 2 pi^2 turns the phase by k |q| = 0.23 rad per step in
    the explicit reaction terms); with k / 4 (320 steps) the GPU is within 0.03
    of the exact solution (oracle: 0.021)."""
    w = W.nls_2d()
    U0 = W.initial_state(w)
    got, _ = gpu_run(w, U0, w.steps)
    ref = oracle.run(oracle_problem(w), U0, 0.0, w.steps)
    e = rel_err(got, ref)
    print(f"nls2d_79 80 steps: gpu vs oracle {e:.2e}")
    assert e <= w.steps * FP64_TOL
    w4 = W.nls_2d(k=w.k / 4)
    got4, _ = gpu_run(w4, U0, w4.steps)
    err_exact = float(np.max(np.abs(got4 - W.exact_nls(w4, w4.steps * w4.k))))
    print(f"nls2d_79 320 steps of k/4: gpu vs exact {err_exact:.3e}")
    assert err_exact < 0.03


def test_cgl_alpha_full_size_one_step_fp32():
    """Section 8's CGL grid (400^2, periodic [0, 200]^2, k = 1/20) with alpha = 0.5:
    one FP32 step against the oracle over the whole grid (its 800 x 800 block
    solves take a few seconds)."""
    w = W.cgl_2d(alpha=0.5, ic="normal")
    U0 = W.initial_state(w)
    got, _ = gpu_run(w, U0, 1, "fp32")
    ref = oracle.run(oracle_problem(w), U0, 0.0, 1)
    e, bound = rel_err(got, ref), fp32_step_bound(w)
    print(f"cgl2d_400_alpha0.5 fp32 1 step: {e:.2e} (bound {bound:.2e})")
    assert e <= bound


def test_coupled_rejections():
    from paper_2001_11220_gb300 import _binding as B
    from paper_2001_11220_gb300.api import EtdRdpIf
    w = CASES[0]
    ctx = EtdRdpIf.from_workload(w, "fp64")
    U = torch.tensor(W.initial_state(w), device="cuda", dtype=torch.float64)
    with pytest.raises(B.EtdError) as ei:
        ctx.grad(U, 0.0, U.clone(), 2, 1)
    assert ei.value.status == B.ETD_ERR_UNSUPPORTED
    with pytest.raises(B.EtdError) as ei:
        ctx.autotune(U.clone())
    assert ei.value.status == B.ETD_ERR_UNSUPPORTED
    ctx.close()


def test_schrodinger_1d_soliton_matches_the_paper_and_the_oracle():
    """Section 8's 1D run on the GPU (d = 1: one fused sweep per step, FP64, 10800 steps):
    the state matches the oracle, and the energy at T = 108 matches the printed value
    to 1e-12, the mass to 5e-11 (the oracle's golden pin, tests/golden/nls1d_soliton.txt)."""
    from paper_2001_11220_gb300.api import EtdRdpIf
    from tests import test_oracle_coupled as C
    g = C.nls1d_golden()
    U0 = C.nls1d_initial()
    nsteps = int(round(C.NLS1D_T / C.NLS1D_K))
    ctx = EtdRdpIf((361,), (W.NEUMANN,), (1.0, 1.0), "nls", (0.0, -1.0, 0.0), C.NLS1D_K, "fp64", (180.0,),
                   Dc=(0.0, -1.0, 1.0, 0.0))
    U = torch.tensor(U0, device="cuda", dtype=torch.float64)
    ctx.run(U, 0.0, nsteps)
    torch.cuda.synchronize()
    info = ctx.info()
    ctx.close()
    got = U.cpu().numpy()
    ref = oracle.run(C.nls1d_problem(), U0, 0.0, nsteps)
    e = rel_err(got, ref)
    print(f"nls1d 10800 steps: gpu vs oracle {e:.2e}, E {C.nls1d_energy(got):.15f}, M {C.nls1d_mass(got):.15f}")
    assert info["launches_per_step"] == 1 and info["staged"][0] == 6
    assert e <= 1e-10
    assert abs(C.nls1d_energy(got) - g[("E", 108)]) < 1e-12
    assert abs(C.nls1d_mass(got) - g[("M", 108)]) < 5e-11


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cgl_alpha_full_size_plane_wave_follows_scalar_recurrence(prec):
    """At the benchmarked 200^3 size (periodic [0, 200]^3, D = 1 + 0.5i, beta = 1.3,
    k = 1/20, the bench's launch configuration) a plane wave a e^{i kappa.x} stays a
    plane wave whose amplitude follows the scalar recurrence of the frame (the
    oracle-pinned closed form of tests/test_oracle_coupled.py): checked on every
    point after 3 steps, FP64 to 1e-12 per step, FP32 within the per-step bound."""
    from tests.test_oracle_coupled import cgl_f, mode_recurrence
    w = W.cgl_3d(200, alpha=0.5)
    ms = (3, 1, 2)
    x = [np.arange(200) * w.h(a) for a in range(3)]
    phase = (2 * math.pi * ms[0] / 200.0) * x[0][None, None, :] + (2 * math.pi * ms[1] / 200.0) * x[1][None, :, None] \
        + (2 * math.pi * ms[2] / 200.0) * x[2][:, None, None]
    a0 = 0.7 * np.exp(0.4j)
    Z0 = a0 * np.exp(1j * phase)
    got, info = gpu_run(w, np.stack([Z0.real, Z0.imag]), 3, prec)
    mus = [4 * math.sin(math.pi * ms[a] / 200.0) ** 2 / w.h(a) ** 2 for a in range(3)]
    an = mode_recurrence(a0, 3, w.k, 1.0 + 0.5j, mus, cgl_f(1.3))
    err = float(np.max(np.abs(got[0] + 1j * got[1] - an * np.exp(1j * phase)))) / abs(an)
    tol = 3 * (FP64_TOL if prec == "fp64" else fp32_step_bound(w))
    print(f"cgl3d_200_alpha0.5 plane wave {prec}: {err:.2e} (tol {tol:.2e}), blocks {info['grid_blocks']}")
    assert info["staged"] == [6, 6, 6]
    assert err <= tol
    assert abs(an - a0) > 1e-3


def test_coupled_host_buffer_run_equals_device_run():
    """etd_run_host (host state, copies inside the call) on a coupled context gives the
    same bits as etd_run on a device state."""
    from paper_2001_11220_gb300.api import EtdRdpIf
    w = CASES[0]
    U0 = W.initial_state(w)
    dev, _ = gpu_run(w, U0, 3)
    ctx = EtdRdpIf.from_workload(w, "fp64")
    H = torch.tensor(U0, dtype=torch.float64).pin_memory()
    ctx.run_host(H, 0.0, 3)
    ctx.close()
    assert np.array_equal(H.numpy(), dev)


def test_line_too_long_for_shared_memory_is_unsupported():
    """A 4000-node FP64 line (4 complex slots: 256 KB) exceeds the kernel's shared
    memory: etd_create_coupled returns ETD_ERR_UNSUPPORTED and allocates nothing."""
    from paper_2001_11220_gb300 import _binding as B
    from paper_2001_11220_gb300.api import EtdRdpIf
    with pytest.raises(B.EtdError) as ei:
        EtdRdpIf((4000, 3), (W.NEUMANN, W.NEUMANN), (1.0, 1.0), "nls", (0.0, -1.0, 0.0), 0.01, "fp64",
                 Dc=(0.0, -1.0, 1.0, 0.0))
    assert ei.value.status == B.ETD_ERR_UNSUPPORTED
    ctx = EtdRdpIf((4000, 3), (W.NEUMANN, W.NEUMANN), (1.0, 1.0), "nls", (0.0, -1.0, 0.0), 0.01, "fp32",
                   Dc=(0.0, -1.0, 1.0, 0.0))   # FP32 slots are half the size: fits
    ctx.close()
