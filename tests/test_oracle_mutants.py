"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a flipped sign, a dropped term, a wrong index, a
transposed operand, a changed rule) in a copy of the oracle's C source, builds
it, and runs the pin suite against it; every mutant must make some pin fail.
The mistakes are planted in the oracle, on the CPU only.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gv_oracle.c")

MUTANTS = {
    "box -x plane flipped": ("set_plane(&s->pl[4], -1, 0, 0, dx);", "set_plane(&s->pl[4], 1, 0, 0, dx);"),
    "tolerance band doubled": ("#define H OR_HALF_TOL", "#define H (2 * OR_HALF_TOL)"),
    "cone normalisation dropped": ("L->k = 1.0 / sqrt(1.0 + L->a * L->a);", "L->k = 1.0;"),
    "section index off by one": ("while (k < s->nz - 2 && z >= s->z[k + 1]) k++;",
                                 "while (k < s->nz - 2 && z >= s->z[k]) k++;"),
    "phi normal sign": ("s->ns[1] = -cos(sphi);", "s->ns[1] = cos(sphi);"),
    "phi wide rule inverted": ("s->phi_wide = dphi > pi;", "s->phi_wide = dphi < pi;"),
    "quadratic root sign": ("const double q = -(B + (B >= 0 ? sq : -sq));",
                            "const double q = -(B - (B >= 0 ? sq : -sq));"),
    "gap classified at its start": ("const double mid = j < m ? 0.5 * (lo + t[j]) : 2.0 * lo + 1.0;",
                                    "const double mid = j < m ? lo : 2.0 * lo + 1.0;"),
    "polycone safety max instead of min": ("best = dmin(best, s_closed(s, k, p));", "best = dmax(best, s_closed(s, k, p));"),
    "trap vertex shear sign": ("const double xm = cx - dy * ta, xp = cx + dy * ta;",
                               "const double xm = cx + dy * ta, xp = cx - dy * ta;"),
    "rotation not transposed": ("pl[i] = (R[0 * 3 + i] * v[0] + R[1 * 3 + i] * v[1]) + R[2 * 3 + i] * v[2];",
                                "pl[i] = (R[i * 3 + 0] * v[0] + R[i * 3 + 1] * v[1]) + R[i * 3 + 2] * v[2];"),
    "daughter tie rule dropped": ("(t == best && who == -1)", "(t == best && who != -1)"),
    "absorption never acts": ("if (proc == 1) { why = OR_ABSORBED; break; }",
                              "if (proc == 2) { why = OR_ABSORBED; break; }"),
    "mean free path inverted": ("-log(r[1]) / sigma_n[2 * m + 1]", "-log(r[1]) * sigma_n[2 * m + 1]"),
    "scatter cosine from the wrong number": ("const double ca = 2.0 * r[2] - 1.0", "const double ca = 2.0 * r[3] - 1.0"),
    "relocation without the push": ("const double q[3] = {p[0] + OR_PUSH * d[0], p[1] + OR_PUSH * d[1], p[2] + OR_PUSH * d[2]};",
                                    "const double q[3] = {p[0], p[1], p[2]};"),
    "boolean union takes the max": ("if (op == OR_UNION) return sa < sc ? sa : sc;", "if (op == OR_UNION) return sa > sc ? sa : sc;"),
    "boolean subtraction keeps c": ("return sa > -sc ? sa : -sc;", "return sa > sc ? sa : sc;"),
    "boolean placement ignored": ("const double v[3] = {p[0] - b->t[0], p[1] - b->t[1], p[2] - b->t[2]};",
                                  "const double v[3] = {p[0], p[1], p[2]};"),
    "boolean union safety max": ("if (to_in) return dmin(sia, sic);", "if (to_in) return dmax(sia, sic);"),
    "trap axis azimuth swapped": ("const double cx = zf * tthc, cy = zf * tths;", "const double cx = zf * tths, cy = zf * tthc;"),
    "trap face quad from the wrong vertices": ("if (face_plane(v[0], v[4], v[6], v[2], cs, &s->pl[4])) return -1;",
                                               "if (face_plane(v[0], v[4], v[7], v[3], cs, &s->pl[4])) return -1;"),
    "section line offset taken at the far plane": ("L->b = r0 - L->a * z0;", "L->b = r0 - L->a * z1;"),
    "tangent threshold dropped": ("#define OR_TAU 1e-12", "#define OR_TAU 0.0"),
    "tangent convex wall entered": ("return outer ? 1 : -1;", "return outer ? -1 : 1;"),
    "generator ray taken as curved": ("if (r > 0 && fabs(p[0] * d[1] - p[1] * d[0]) > OR_TAU * r)", "if (r > 0)"),
    "sliding surfaces not detected": ("if (fabs(c[i].g) <= H && c[i].m == 0) sl->bits |= c[i].bit;",
                                      "if (0) sl->bits |= c[i].bit;"),
    "sliding counted as inside": ("slide_setup1(s, p, d, INFINITY, &sl->a);", "slide_setup1(s, p, d, -INFINITY, &sl->a);"),
    "subtracted face slide counted as outside c": ("s->bl->op == OR_SUBTRACTION ? -INFINITY : INFINITY", "INFINITY"),
    "double root taken as a crossing": ("if (disc > OR_DISC * ((fabs(B) * Bs + fabs(A) * Cs) + fabs(C) * As))",
                                        "if (disc > 0)"),
    "crossings not merged": ("#define OR_MERGE 1e-12", "#define OR_MERGE 0.0"),
    "surface start leaves only when a constraint grows": (
        "if (c[i].motion && c[i].g >= -H && c[i].m != -1) return 0;",
        "if (c[i].motion && c[i].g >= -H && c[i].m == 1) return 0;"),
    "boundary step shortened": ("for (int j = 0; j < 3; j++) p[j] = p[j] + dgeo * d[j];",
                                "for (int j = 0; j < 3; j++) p[j] = p[j] + 0.5 * dgeo * d[j];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {name}"
    mutated = src.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "gv_oracle.c")
        open(c, "w").write(mutated)
        with open(os.path.join(ROOT, "oracle", "gv_oracle.h")) as h:
            open(os.path.join(d, "gv_oracle.h"), "w").write(h.read())
        so = os.path.join(d, "mutant.so")
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", c,
                        "-o", so, "-lm"], check=True)
        env = dict(os.environ, GV_ORACLE_SO=so, GV_ORACLE_THREADS="4")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutant '{name}' survived the pins"
