"""Planted mistakes in the oracle must be caught by its pins.

(Two natural-looking mutations are deliberately absent because they are
equivalent: negating every s-interface reflection coefficient maps the product
to diag(1, -1) M diag(1, -1), which leaves R and T unchanged -- the same sign
freedom that makes r_p = -r_s at normal incidence; and keeping the slope of a
clamped Im(delta) changes the gradient only by terms of order e^-70.)

Each mutant is a copy of ``oracle/tmm_oracle.c`` with one plausible error (a
swapped phase factor, a sign, a transposed product, a wrong index or
conjugation, a dropped term), compiled on the CPU; the battery below -- the
same kinds of closed forms, invariants and cross-checks as the pins -- must
flag every mutant and pass the unmodified oracle."""
import numpy as np
import pytest

import oracle
from oracle.admittance import coh_tmm_admittance
from tests.helpers import stack

MUTANTS = {
    "phase factors swapped": ("cplx em = cexp(-I * delta), ep = cexp(I * delta);",
                              "cplx em = cexp(I * delta), ep = cexp(-I * delta);"),
    "s reflection uses one angle": ("        *r = (n1 * c1 - n2 * c2) / den;\n        *t = 2.0 * n1 * c1 / den;\n    } else {",
                                    "        *r = (n1 * c1 - n2 * c1) / den;\n        *t = 2.0 * n1 * c1 / den;\n    } else {"),
    "r extracted from the wrong entry": ("    cplx r = M.c / M.a;", "    cplx r = M.b / M.a;"),
    "p uses the s denominator": ("        cplx den = n2 * c1 + n1 * c2;\n        *r = (n2 * c1 - n1 * c2) / den;",
                                 "        cplx den = n1 * c1 + n2 * c2;\n        *r = (n2 * c1 - n1 * c2) / den;"),
    "product order transposed": ("        M = mat2_mul(M, Mj);", "        M = mat2_mul(Mj, M);"),
    "phase uses next medium": ("cplx delta = 2.0 * M_PI * nj * d[j - 1] * c[j] / lambda;",
                               "cplx delta = 2.0 * M_PI * nj * d[j - 1] * c[j + 1] / lambda;"),
    "clamp too low": ("#define ORACLE_IM_DELTA_MAX 35.0", "#define ORACLE_IM_DELTA_MAX 3.5"),
    "T_p without conjugates": ("T = creal(nout * conj(c[L + 1])) / creal(nin * conj(c[0])) * creal(t * conj(t));",
                               "T = creal(nout * c[L + 1]) / creal(nin * c[0]) * creal(t * conj(t));"),
    "t_s from the wrong medium": ("        *r = (n1 * c1 - n2 * c2) / den;\n        *t = 2.0 * n1 * c1 / den;",
                                  "        *r = (n1 * c1 - n2 * c2) / den;\n        *t = 2.0 * n2 * c2 / den;"),
    "Snell multiplies": ("    cplx s = beta / n;", "    cplx s = beta * n;"),
    "grazing reading dropped": ("    if (c[0] == 0.0) { /* exact grazing incidence */",
                                "    if (0) { /* exact grazing incidence */"),
    "root choice ignores decay": ("    } else if (cimag(nc) < 0.0) {\n        c = -c;\n    }",
                                  "    } else if (cimag(nc) > 0.0) {\n        c = -c;\n    }"),
    "gradient of the root": ("if (n.e != 0.0) r.e = beta * beta * n.e / (n.v * n.v * n.v * c);",
                             "if (n.e != 0.0) r.e = beta * beta * n.e / (n.v * n.v * c);"),
    "dual phase misses the index": ("dual delta = dscale(2.0 * M_PI / lambda, dmul(dmul(nn[j], dj), c[j]));",
                                    "dual delta = dscale(2.0 * M_PI / lambda, dmul(dj, c[j]));"),
}

LAM = np.linspace(420.0, 880.0, 17)
TH = np.deg2rad([0.0, 35.0, 70.0])


def _random(rng, L, absorbing, sub=1.52):
    n = np.empty((3, L + 2), dtype=np.complex128)
    n[:, 0] = 1.0
    n[:, 1:L + 1] = rng.uniform(1.3, 2.6, (3, L)) + (1j * rng.uniform(0.0, 0.3, (3, L)) if absorbing else 0)
    n[:, L + 1] = sub
    return np.repeat(n[:, :, None], LAM.size, axis=2), rng.uniform(5, 400, (3, L))


def battery(lib):
    """Names of the checks this build of the oracle fails."""
    fails = []
    rng = np.random.default_rng(5)

    def check(name, ok):
        if not ok:
            fails.append(name)

    # quarter-wave closed form, normal incidence
    media = [1.0] + [2.35, 1.46] * 3 + [1.52]
    dq = [600 / (4 * 2.35), 600 / (4 * 1.46)] * 3
    Y = (2.35 / 1.46) ** 6 * 1.52
    n, d = stack(media, dq)
    for pol in "sp":
        R, _ = oracle.coh_tmm(pol, n, d, [0.0], [600.0], lib=lib)
        check("quarter-wave", np.isfinite(R).all() and abs(R[0, 0, 0] - ((1 - Y) / (1 + Y)) ** 2) < 1e-12)
    # Brewster
    n, d = stack([1.0, 1.5], [])
    R, _ = oracle.coh_tmm("p", n, d, [np.arctan(1.5)], [600.0], lib=lib)
    check("brewster", np.isfinite(R).all() and R[0, 0, 0] < 1e-25)
    # lossless R + T = 1 and an absorbing, metal-backed stack against the admittance form
    nn, dd = _random(rng, 9, absorbing=False)
    for pol in "sp":
        R, T = oracle.coh_tmm(pol, nn, dd, TH, LAM, lib=lib)
        check("R+T=1", np.isfinite(R).all() and np.max(np.abs(R + T - 1)) < 1e-12)
    for sub in (1.52, 0.3 + 2.5j):
        nn, dd = _random(rng, 7, absorbing=True, sub=sub)
        for pol in "sp":
            R, T = oracle.coh_tmm(pol, nn, dd, TH, LAM, lib=lib)
            good = np.isfinite(R).all() and np.isfinite(T).all()
            for s in range(nn.shape[0]):
                Ra, Ta = coh_tmm_admittance(pol, nn[s], dd[s], TH, LAM)
                good = good and np.max(np.abs(R[s] - Ra)) < 1e-11 and np.max(np.abs(T[s] - Ta)) < 1e-11
            check("admittance", good)
    # opaque layer: only the front interface is seen; many opaque layers stay finite
    for pol in "sp":
        n, d = stack([1.0, 2 + 1j, 1.7, 1.52], [1e5, 80.0], n_lambda=LAM.size)
        R, _ = oracle.coh_tmm(pol, n, d, TH, LAM, lib=lib)
        nb, db = stack([1.0, 2 + 1j], [], n_lambda=LAM.size)
        Rb, _ = oracle.coh_tmm(pol, nb, db, TH, LAM, lib=lib)
        check("opaque", np.isfinite(R).all() and np.max(np.abs(R - Rb)) < 1e-13)
        n, d = stack([1.0] + [2 + 1j, 1.5] * 15 + [1.52], [1e5, 90.0] * 15, n_lambda=LAM.size)
        R, T = oracle.coh_tmm(pol, n, d, TH, LAM, lib=lib)
        check("opaque-finite", np.isfinite(R).all() and np.isfinite(T).all())
        # grazing
        n, d = stack([1.0, 1.8, 1.52], [100.0])
        R, T = oracle.coh_tmm(pol, n, d, [np.pi / 2], [500.0], lib=lib)
        check("grazing", R[0, 0, 0] == 1.0 and T[0, 0, 0] == 0.0)
    # total internal reflection: R = 1 with an evanescent outcoupling medium
    n, d = stack([1.5, 1.8, 1.0], [120.0], n_lambda=LAM.size)
    R, T = oracle.coh_tmm("s", n, d, np.deg2rad([50.0, 70.0]), LAM, lib=lib)
    check("tir", np.isfinite(R).all() and np.max(np.abs(R - 1)) < 1e-12 and np.max(np.abs(T)) < 1e-12)
    # gradient against central differences (one stack, including a clamped opaque layer)
    nn = np.array([[1.0, 1.9 + 0.05j, 2.0 + 1.0j, 1.6, 1.52]], dtype=np.complex128)
    nn = np.repeat(nn[:, :, None], 5, axis=2)
    dd = np.array([[80.0, 2e4, 120.0]])
    lam = np.linspace(450, 750, 5)
    th = np.deg2rad([0.0, 40.0])
    Rt = np.full((2, 2, 5), 0.3)
    _, gd, gn = oracle.merit_grad("sp", nn, dd, th, lam, Rt, lib=lib)
    f = lambda n_, d_: oracle.merit("sp", n_, d_, th, lam, Rt, lib=lib)
    good = True
    for j in range(3):
        dp, dm = dd.copy(), dd.copy()
        dp[0, j] += 1e-4
        dm[0, j] -= 1e-4
        fd = (f(nn, dp) - f(nn, dm)) / 2e-4
        good = good and abs(fd[0] - gd[0, j]) <= 1e-6 * max(1e-12, abs(fd[0])) + 1e-12
        npl, nmi = nn.copy(), nn.copy()
        npl[0, j + 1] += 1e-6
        nmi[0, j + 1] -= 1e-6
        fd = (f(npl, dd) - f(nmi, dd)) / 2e-6
        good = good and abs(fd[0] - gn[0, j]) <= 1e-5 * max(1e-12, abs(fd[0])) + 1e-10
    check("gradient", good)
    return fails


def test_unmodified_oracle_passes_battery():
    assert battery(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, f"mutation site of {name!r} not unique"
    lib = oracle.build_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    fails = battery(lib)
    assert fails, f"mutant {name!r} survived every check"
