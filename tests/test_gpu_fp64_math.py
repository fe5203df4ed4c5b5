"""The fill's FP64 device routines against CUDA's library functions and the oracle.

  * square root (FP32 seed + two Newton steps): within 1 ulp of the correctly rounded
    sqrt (torch.sqrt on the device); reciprocal square root: within 2 ulp of 1/sqrt;
  * exp(-x) (table-driven reduction after Tang, 1989): within 2 ulp of CUDA's exp
    (torch.exp on the device) and of the host's exp, and 0 below -700;
  * the Matern at squared distance d2: within (6 + 3t) * 2^-52 relative of the oracle's
    FP64 Matern (t = sqrt(2 nu) r / ell; the two sides round t differently by up to ~2
    ulp, and an ulp of t moves exp(-t) by t ulp).
"""
import math

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11648_gb300 import build
    build.build()
    from paper_2307_11648_gb300 import sic
    return torch, sic, sic.Handle(0)


def _inputs(torch):
    u = synthetic.uniform(71, 0, 200000)
    x = np.concatenate([
        np.exp(np.log(1e-36) + u[:50000] * (np.log(1e36) - np.log(1e-36))),  # log-uniform 1e-36 .. 1
        u[50000:150000] * 40.0,                                              # the Matern range
        u[150000:] * 750.0,                                                  # up to the cut-off
        [0.0, 1e-40, 2.0 ** -120, 1.0, 4.0, 699.9, 700.0, 700.5, 1e30, 1e40],
    ])
    return torch.tensor(x, dtype=torch.float64, device="cuda"), x


def test_sqrt_and_exp_against_cuda(env):
    torch, sic, h = env
    kp = sic.kernel(2, 3, 0.1, 1.0, 0.0)
    xt, x = _inputs(torch)
    s, rs, e, _ = sic.selftest_fp64_math(h, kp, xt)
    h.sync()
    s = s.cpu().numpy()
    rs = rs.cpu().numpy()
    e = e.cpu().numpy()
    s_ref = torch.sqrt(xt).cpu().numpy()
    ok = x >= 2.0 ** -120
    assert np.all(s[~ok] == 0.0)
    rel = np.abs(s[ok] - s_ref[ok]) / s_ref[ok]
    print("sqrt max rel err", rel.max() / ULP, "ulp")
    assert rel.max() <= ULP
    pos = x > 0
    r_ref = (1.0 / torch.sqrt(xt)).cpu().numpy()
    rrel = np.abs(rs[pos] - r_ref[pos]) / r_ref[pos]
    print("rsqrt max rel err", rrel.max() / ULP, "ulp")
    assert rrel.max() <= 2 * ULP
    e_cuda = torch.exp(-xt).cpu().numpy()
    e_host = np.exp(-x)
    live = x <= 700.0
    assert np.all(e[~live] == 0.0)
    for ref, name in [(e_cuda, "cuda"), (e_host, "host")]:
        r = np.abs(e[live] - ref[live]) / ref[live]
        print(f"exp max rel err vs {name}", r.max() / ULP, "ulp")
        assert r.max() <= 2 * ULP


@pytest.mark.parametrize("nu_x2", [1, 3, 5])
def test_matern_against_oracle(env, oracle_lib, nu_x2):
    torch, sic, h = env
    ell, s2 = 0.07, 1.7
    kp = sic.kernel(3, nu_x2, ell, s2, 0.0)
    d2 = synthetic.uniform(72, nu_x2, 100000) * (20 * ell) ** 2
    d2[:3] = [0.0, 1e-30, ell * ell]
    _, _, _, kv = sic.selftest_fp64_math(h, kp, torch.tensor(d2, dtype=torch.float64, device="cuda"))
    h.sync()
    kv = kv.cpu().numpy()
    okp = oracle_lib.kernel(3, nu_x2, ell, s2, 0.0)
    r = np.sqrt(d2)
    ref = np.array([oracle_lib.matern(okp, v) for v in r])
    t = math.sqrt(nu_x2) * r / ell
    err = np.abs(kv - ref) / (ref * (6 + 3 * t) * ULP)
    print(f"nu={nu_x2}/2 Matern max err / ((6 + 3t) ulp)", err.max())
    assert err.max() <= 1.0


@pytest.mark.parametrize("dim,nu_x2,ell,variance", [(2, 3, 0.02, 1.0), (3, 5, 0.05, 1.0), (2, 1, 0.1, 2.5),
                                                    (2, 3, 0.1, 1.0)])
def test_double_float_matern_against_the_oracle(env, oracle_lib, dim, nu_x2, ell, variance):
    """The fill's double-float Matern (dfloat.cuh: coordinates relative to an origin as
    double-floats, distance, square root and table-driven exponential in double-float on
    the FP32 pipe) against the oracle's FP64 Matern (C, libm exp) on point pairs at
    distances from 1e-7 ell to 40 ell, coordinates in the unit cube: the absolute error
    must stay below 2e-14 of the variance.  Basis: each double-float addition or product
    carries a relative error of at most about 3 * 2^-48 (its one rounded FP32 operation on
    the low parts), and an entry passes through about eight of them after the distance
    (square root, t, the reduction, e^r - 1, the table product, the Matern polynomial), so
    about 1e-14 of the entry (an emulation of the same operations in numpy measured 9e-15
    worst over 60,000 pairs); the FP64 fill needs this much: its entries' errors enter the
    factorisation as a perturbation of Theta of that absolute size (the fill's parity bar
    is 1e-8 of a column, with effective condition numbers up to ~1e5 measured here)."""
    torch, sic, h = env
    kp = sic.kernel(dim, nu_x2, ell, variance, 0.0)
    n = 200000
    pa = synthetic.uniform(81, 0, n * dim).reshape(n, dim)
    direc = synthetic.normal(82, n * dim).reshape(n, dim)
    direc /= np.linalg.norm(direc, axis=1, keepdims=True)
    u = synthetic.uniform(83, 0, n)
    r = ell * np.exp(np.log(1e-7) + u * (np.log(40.0) - np.log(1e-7)))
    pb = pa + direc * r[:, None]
    got = sic.selftest_matern_df(h, kp, torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()).cpu().numpy()
    h.sync()
    okp = oracle_lib.kernel(dim, nu_x2, ell, variance, 0.0)
    ref = np.array([oracle_lib.matern(okp, float(np.linalg.norm(b - a))) for a, b in zip(pa, pb)])
    err = np.abs(got - ref)
    print(f"dim {dim} nu {nu_x2}/2 ell {ell}: max abs err {err.max() / variance:.3e} of the variance, "
          f"max rel err where the entry > 1e-3: {np.max(err[ref > 1e-3 * variance] / ref[ref > 1e-3 * variance]):.3e}")
    assert err.max() <= 2e-14 * variance


@pytest.mark.parametrize("dim", [2, 3])
def test_fixed_point_routines_against_exact_rationals(env, dim):
    """The fill's integer arithmetic: squared distances from fixed-point coordinates must be the
    correctly rounded exact value (0.5 ulp; differences and squares are exact in 128 bits), and
    the panels' 4-term dot products of fixed-point rows within 12 * 2^-52 max|a| max|b| of the
    exact sum (each value truncated below 2^-52 of its row's largest, the sum below 2^-51 of
    the largest product)."""
    from fractions import Fraction as F
    torch, sic, h = env
    n = 20000
    u = synthetic.uniform(91, dim, n * dim).reshape(n, dim)
    direc = synthetic.normal(92, n * dim).reshape(n, dim)
    sep = np.exp(np.log(1e-9) + synthetic.uniform(93, 0, n) * (np.log(1.0) - np.log(1e-9)))
    pa = u
    pb = u + direc * sep[:, None]
    pb[::17] = pa[::17]                     # coincident points
    pa[::29, 0] = 3e-6 * synthetic.uniform(94, 0, len(pa[::29]))   # coordinates near zero
    pb[::29, 0] = pa[::29, 0] + 1e-7
    g = synthetic.normal(95, n * 8).reshape(n, 8)
    mag = np.exp(np.log(1e-12) + synthetic.uniform(96, 0, n * 8).reshape(n, 8) * (np.log(10.0) - np.log(1e-12)))
    g = g * mag
    g[::13, 1] = 0.0
    ga, gb = g[:, :4].copy(), g[:, 4:].copy()
    d2, dot = sic.selftest_fixed_point(h, torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda(),
                                       torch.from_numpy(ga).cuda(), torch.from_numpy(gb).cuda())
    h.sync()
    d2 = d2.cpu().numpy()
    dot = dot.cpu().numpy()
    worst_d2 = worst_dot = 0.0
    for i in range(n):
        ex = sum((F(float(a)) - F(float(b))) ** 2 for a, b in zip(pa[i], pb[i]))
        if ex == 0:
            assert d2[i] == 0.0
        else:
            worst_d2 = max(worst_d2, float(abs(F(float(d2[i])) - ex) / F(math.ulp(float(ex)))))
        exd = sum(F(float(a)) * F(float(b)) for a, b in zip(ga[i], gb[i]))
        bound = 12 * 2.0 ** -52 * np.max(np.abs(ga[i])) * np.max(np.abs(gb[i]))
        err = float(abs(F(float(dot[i])) - exd))
        worst_dot = max(worst_dot, err / bound if bound > 0 else (0.0 if err == 0 else math.inf))
    print(f"dim {dim}: d2 worst {worst_d2:.3f} ulp; dot worst {worst_dot:.3f} of the bound")
    assert worst_d2 <= 0.5
    assert worst_dot <= 1.0
