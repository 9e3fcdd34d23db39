"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped term, a wrong
sign, a swapped index, an unstable sort, ...), builds it on the CPU and runs the pins that
should catch it against the broken build, expecting at least one failure.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mpcd_oracle.c")

MUTANTS = [
    ("rotation sense flipped", "out[k] = par * n[k] + c * perp + s * cr[k];",
     "out[k] = par * n[k] + c * perp - s * cr[k];", "rotation"),
    ("parallel part dropped", "out[k] = par * n[k] + c * perp + s * cr[k];",
     "out[k] = c * perp + s * cr[k];", "rotation"),
    ("rotation about v instead of v - u", "d[k] = v[k] - u[k];", "d[k] = v[k];", "galilean or conserves"),
    ("mass weight dropped", "P[d] += mi * vi[d];", "P[d] += vi[d];", "closed_form or conserves or mass"),
    ("key index order swapped", "return c[0] + (int64_t)p->L[0] * (c[1] + (int64_t)p->L[1] * c[2]);",
     "return c[1] + (int64_t)p->L[1] * (c[0] + (int64_t)p->L[0] * c[2]);", "brute_force or face_point"),
    ("shift sign flipped", "double q = (r[d] - s[d]) / p->a;\n    int64_t k = (int64_t)floor(q);",
     "double q = (r[d] + s[d]) / p->a;\n    int64_t k = (int64_t)floor(q);",
     "brute_force or face_point"),
    ("perm not stable", "for (int64_t i = 0; i < n; ++i) perm[cur[key[i]]++] = (int32_t)i;",
     "for (int64_t i = n - 1; i >= 0; --i) perm[cur[key[i]]++] = (int32_t)i;", "stable_argsort"),
    ("philox key schedule skipped", "k0 += PHILOX_W0;", "k0 += 0;", "kat or numpy"),
    ("philox words swapped", "uint64_t y1 = lo1;", "uint64_t y1 = lo0;", "kat or numpy"),
    ("no streaming", "r[d] = fma(v[d], p->dt, r[d] + h);", "r[d] = r[d] + h;", "streaming"),
    ("axis not uniform", "double z = 2.0 * orc_u53(w[0]) - 1.0;", "double z = orc_u53(w[0]);", "axis_uniform"),
    ("wall bounce keeps velocity", "for (int d = 0; d < 3; ++d) v[d] = -v[d];",
     "for (int d = 2; d < 3; ++d) v[d] = -v[d];", "bounce_back"),
    ("gamma shift d without the 1/3", "double d = shape - 1.0 / 3.0;", "double d = shape;", "mbs"),
    ("gamma cube dropped", "double v = tt * tt * tt;", "double v = tt * tt;", "mbs"),
    ("gamma squeeze too loose", "if (u < 1.0 - 0.0331 * (x2 * x2)) return d * v;",
     "if (u < 1.0 - 0.00331 * (x2 * x2)) return d * v;", "mbs"),
    ("MBS shape from n_c instead of n_c - 1", "orc_mbs_gamma(p, t, c, 1.5 * (double)(nc - 1))",
     "orc_mbs_gamma(p, t, c, 1.5 * (double)nc)", "mbs"),
    ("MBS target without kT", "? p->kT * orc_mbs_gamma(", "? orc_mbs_gamma(", "mbs"),
    ("angular correction sign flipped", "for (int d = 0; d < 3; ++d) vi[d] += corr[d];",
     "for (int d = 0; d < 3; ++d) vi[d] -= corr[d];", "angular or omega or two_particle"),
    ("inertia tensor without the |rho|^2 term", "I[a][b] += mi * ((a == b ? q2 : 0.0) - q[a] * q[b]);",
     "I[a][b] += mi * (0.0 - q[a] * q[b]);", "angular or omega or two_particle"),
    ("positions not taken about the centre of mass", "= p->a * (rc[3 * (int64_t)(j - off[c]) + d] - mean[d]);",
     "= p->a * (rc[3 * (int64_t)(j - off[c]) + d] - 0.0 * mean[d]);", "angular or omega or two_particle"),
    ("two-particle omega off by two", "w[d] = (dL[d] - along * q[d]) / (p->mass * rr);",
     "w[d] = (dL[d] - along * q[d]) / (2.0 * p->mass * rr);", "angular or omega or two_particle"),
    ("cell mass counts particles", "      M += mi;\n", "      M += 1.0;\n", "mass"),
    ("thermostat energy unweighted", "K += 0.5 * mi * (vi[d] - u[d]) * (vi[d] - u[d]);",
     "K += 0.5 * (vi[d] - u[d]) * (vi[d] - u[d]);", "mass"),
    ("masses left behind on re-sort", "m2[j] = mass ? mass[i] : 0.0;", "m2[j] = mass ? mass[j] : 0.0;", "mass"),
    ("centre of mass unweighted", "mean[d] += mass ? mass[perm[j]] * l[d] : l[d];", "mean[d] += l[d];", "mass"),
    ("virtual mass left out of the cell mass", "        M += Mv;\n", "        M += 0.0;\n", "virtual"),
    ("virtual momentum variance without the mass", "double sd = sqrt(Mv * p->kT);",
     "double sd = sqrt(Mv * p->kT / m);", "virtual"),
    ("virtual momentum variance from the real particles", "double sd = sqrt(Mv * p->kT);",
     "double sd = sqrt((double)nc * m * p->kT);", "virtual"),
    ("virtual fill in every layer", "if ((layer == 0 || layer == p->L[2]) && (double)nc < p->ppc) {",
     "if ((double)nc < p->ppc) {", "virtual"),
    ("virtual fill in the wrong wall layer", "if ((layer == 0 || layer == p->L[2]) && (double)nc < p->ppc) {",
     "if ((layer == 0 || layer == p->L[2] - 1) && (double)nc < p->ppc) {", "virtual"),
    ("virtual fill count rounded down", "double Mv = (p->ppc - (double)nc) * m;",
     "double Mv = (floor(p->ppc) - (double)nc) * m;", "virtual"),
    ("virtual momentum on the axis stream", "draw(p, (uint64_t)t, (uint64_t)c, ORC_TAG_WALL, w);",
     "draw(p, (uint64_t)t, (uint64_t)c, ORC_TAG_AXIS, w);", "virtual"),
    ("presort not stable", "for (int64_t i = 0; i < n; ++i) order[start[key[i]]++] = i;",
     "for (int64_t i = n - 1; i >= 0; --i) order[start[key[i]]++] = i;", "presort"),
    ("presort on the shifted grid", "const double s0[3] = {0.0, 0.0, 0.0};",
     "const double s0[3] = {0.25, 0.0, 0.0};", "presort"),
    ("cofactor indices swapped", "cof[a][b] = I[a1][b1] * I[a2][b2] - I[a1][b2] * I[a2][b1];",
     "cof[a][b] = I[a1][b1] * I[a2][b2] - I[a1][b2] * I[a1][b2];", "angular or omega or two_particle"),
]


@pytest.mark.parametrize("name,old,new,select", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new, select):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found: " + name
    mutated = tmp_path / "mpcd_oracle.c"
    mutated.write_text(src.replace(old, new))
    (tmp_path / "mpcd_oracle.h").write_text(open(SRC[:-2] + ".h").read())
    lib = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib),
                    str(mutated), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    tests = [os.path.join(ROOT, "tests", f) for f in
             ("test_oracle_philox.py", "test_oracle_geometry.py", "test_oracle_rotation.py",
              "test_oracle_step.py", "test_oracle_walls.py", "test_oracle_thermostat.py",
              "test_oracle_angular.py", "test_oracle_masses.py")]
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          "-k", select + " and not poiseuille and not relaxes"] + tests,
                         cwd=ROOT, env=env, capture_output=True, text=True)
    assert res.returncode == 1, "mutant survived: %s\n%s" % (name, res.stdout[-2000:])
