"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of ``oracle/sbg_oracle.c`` (a dropped term, a wrong sign, index,
spacing or operand), builds it into a separate library under ``_build/`` and
runs the oracle pin files against it in a child process (SBG_ORACLE_LIB);
at least one pin must fail.  The real oracle is never modified."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sbg_oracle.c")
OUT = os.path.join(ROOT, "_build", "oracle_mutants")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_inhom.py", "tests/test_oracle_sussman.py",
        "tests/test_oracle_frap.py"]

# (name, text in the oracle, planted replacement); the text must occur once
MUTANTS = [
    ("mirror dropped: an inactive neighbour reads 0",
     "return active[j] ? u[j] : uc;", "return active[j] ? u[j] : 0.0;"),
    ("box edge not mirrored",
     "if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) return uc;",
     "if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) return 0.0;"),
    ("second difference with a wrong sign",
     "lap += coef * ((up - uc) - (uc - um));", "lap += coef * ((up - uc) + (uc - um));"),
    ("x spacing used on every axis",
     "double coef = (lap_only ? 1.0 : D[s]) / (dx[a] * dx[a]);",
     "double coef = (lap_only ? 1.0 : D[s]) / (dx[0] * dx[0]);"),
    ("surface transfer uses the species' own value instead of A's",
     "k_surf * w[i] * u[i] : 0.0;", "k_surf * w[i] * us[i] : 0.0;"),
    ("species B loses the transfer instead of gaining it",
     "else if (s == 1) react += transfer;", "else if (s == 1) react -= transfer;"),
    ("decay with the wrong sign",
     "double react = -decay[s] * uc;", "double react = decay[s] * uc;"),
    ("Dirichlet-held voxels updated",
     "if (fixed[i]) { u_next[si] = u[si]; continue; }", "(void)0;"),
    ("flux with the y spacing",
     "double j = D[s] * (us[i] - us[i + 1]) / dx[0] * area;",
     "double j = D[s] * (us[i] - us[i + 1]) / dx[1] * area;"),
    ("residual without the square root",
     "out[s * 5 + 3] = sqrt(sum_slices(part + 3 * nz, nz));",
     "out[s * 5 + 3] = sum_slices(part + 3 * nz, nz);"),
    ("inactive voxels counted in the reductions",
     "if (!active[i]) continue;\n                    kadd(&cnt, 1.0);", "kadd(&cnt, 1.0);"),
    ("stability limit without the factor 2",
     "double rate = 2.0 * D[s] * inv2 + decay[s];", "double rate = D[s] * inv2 + decay[s];"),
    ("surface weight twice the unit delta",
     "(1.0 + cos(pi * p / band_eps)) / (2.0 * band_eps)", "(1.0 + cos(pi * p / band_eps)) / band_eps"),
    ("adjoint coupling not transposed",
     "if (s == 0 && nspecies == 2) val += dt * k_surf * wi * lam_next[n + i];",
     "if (s == 1 && nspecies == 2) val += dt * k_surf * wi * lam_next[i];"),
    ("adjoint takes held neighbours' lambda",
     "if (!fixed[j]) off += c * ls[j];", "off += c * ls[j];"),
    ("dL/dk with the wrong sign",
     "kadd(&gk, dt * wi * u_n[i] * (lb - lam_next[i]));", "kadd(&gk, dt * wi * u_n[i] * (lam_next[i] - lb));"),
    ("face diffusivity from the neighbour only",
     "const double dp = D * (ec + ep) / 2.0, dm = D * (ec + em) / 2.0;",
     "const double dp = D * ep, dm = D * em;"),
    ("Eq. 6 sigmoid with the wrong sign",
     "exp(-(g1 + g2 * (double)phi[i]))", "exp(g1 + g2 * (double)phi[i])"),
    ("upwind branch of phi > 0 taken from the wrong side",
     "s1 = dm > 0.0 ? dm : 0.0;", "s1 = dm < 0.0 ? dm : 0.0;"),
    ("redistancing moves away from |grad phi| = 1",
     "out[IDX(x, y, z)] = c + dalpha * sigma * (1.0 - g);", "out[IDX(x, y, z)] = c + dalpha * sigma * (g - 1.0);"),
    ("box sum over inactive voxels",
     "if (!active[i]) continue;\n                kadd(&m, u[i]);", "kadd(&m, u[i]);"),
    ("D_eff over the box length N dx instead of the distance (N - 1) dx between the held planes",
     "const double L = (double)(dims[0] - 1) * dx[0];", "const double L = (double)dims[0] * dx[0];"),
    ("tau without the porosity",
     "*tau = (*D_eff > 0.0) ? (*psi) * D / (*D_eff) : INFINITY;", "*tau = (*D_eff > 0.0) ? D / (*D_eff) : INFINITY;"),
    ("inhomogeneous flux with the centre's factor only",
     "const double j = D * (eps[i] + eps[i + 1]) / 2.0 * (u[i] - u[i + 1]) / dx[0] * area;",
     "const double j = D * eps[i] * (u[i] - u[i + 1]) / dx[0] * area;"),
    ("inhomogeneous update without decay",
     "return lap - decay * uc;", "return lap;"),
    ("dL/dD from the full right-hand side instead of the Laplacian",
     "decay, k_surf, 1);", "decay, k_surf, 0);"),
    ("external source subtracted instead of added",
     "if (src) r += src[si];", "if (src) r -= src[si];"),
    ("steady-state operator with the x spacing on every axis",
     "(dx[a] * dx[a]) * (eps ? 0.5 * (eps[i] + eps[j]) : 1.0);\n                        /* held",
     "(dx[0] * dx[0]) * (eps ? 0.5 * (eps[i] + eps[j]) : 1.0);\n                        /* held"),
    ("steady-state operator with the neighbour's factor only",
     "(dx[a] * dx[a]) * (eps ? 0.5 * (eps[i] + eps[j]) : 1.0);\n                        /* held",
     "(dx[a] * dx[a]) * (eps ? eps[j] : 1.0);\n                        /* held"),
    ("active set includes phi equal to the threshold",
     "active[i] = (phi[i] > eps_mask) ? 1 : 0;", "active[i] = (phi[i] >= eps_mask) ? 1 : 0;"),
    ("Dirichlet mask on the wrong x face",
     "(dirichlet[1] && x == nx - 1)", "(dirichlet[1] && x == nx - 2)"),
    ("surface weight outside the band",
     "(active[i] && p < band_eps)", "(active[i] && p <= 2.0 * band_eps)"),
    ("stability limit without the surface rate",
     "if (s == 0 && k_surf > 0.0) rate += k_surf / band_eps;", "(void)0;"),
    ("inlet flux at the wrong plane",
     "if (x == 0) kadd(&jin, j);\n                        if (x == nx - 2) kadd(&jout, j);\n                    }\n"
     "                }\n            part[0 * nz + z] = m.s;",
     "if (x == 1) kadd(&jin, j);\n                        if (x == nx - 2) kadd(&jout, j);\n                    }\n"
     "                }\n            part[0 * nz + z] = m.s;"),
    ("adjoint diagonal without the reaction rate",
     "double diag = 1.0 - dt * sum_c - dt * rate;", "double diag = 1.0 - dt * sum_c;"),
    ("smoothed sign without the gradient term",
     "const double sigma = c / sqrt(c * c + g * g * h * h);", "const double sigma = c / sqrt(c * c + h * h);"),
    ("voxels with phi = 0 updated by the redistancing",
     "if (c == 0.0) {\n                        out[IDX(x, y, z)] = c;\n                        continue;\n                    }", ""),
    ("adjoint keeps lambda on held voxels",
     "if (!active[i] || fixed[i]) {\n                    for (int s = 0; s < nspecies; ++s) lam_n",
     "if (!active[i]) {\n                    for (int s = 0; s < nspecies; ++s) lam_n"),
]


def _build(idx, text, repl):
    src = open(SRC).read()
    if text is None:  # the oracle as it is
        text = repl = src
    assert src.count(text) == 1, "mutation site %d not found once in the oracle" % idx
    os.makedirs(OUT, exist_ok=True)
    c = os.path.join(OUT, "mutant%02d.c" % idx)
    so = os.path.join(OUT, "mutant%02d.so" % idx)
    open(c, "w").write(src.replace(text, repl))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", c, "-o", so,
                    "-lm"], check=True, capture_output=True)
    return so


def _run_pins(so):
    env = dict(os.environ, SBG_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "--timeout", "120"] + PINS, cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    return r.returncode, (r.stdout + r.stderr)[-600:]


def test_every_planted_mistake_fails_a_pin():
    with ThreadPoolExecutor(max_workers=4) as ex:
        libs = list(ex.map(lambda a: _build(*a), [(i, t, r) for i, (_, t, r) in enumerate(MUTANTS)]))
        results = list(ex.map(_run_pins, libs))
    survived = [(MUTANTS[i][0], tail) for i, (rc, tail) in enumerate(results) if rc == 0]
    assert not survived, survived
    # a pin failed, not the collection or the loader
    for i, (rc, tail) in enumerate(results):
        assert rc == 1, (MUTANTS[i][0], rc, tail)


def test_the_unmodified_oracle_passes_through_the_same_harness():
    so = _build(99, None, None)
    rc, tail = _run_pins(so)
    assert rc == 0, tail
