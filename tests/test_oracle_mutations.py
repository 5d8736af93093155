"""Each planted mistake in a copy of the oracle must fail at least one pin.

The mistakes are the plausible ones for this method: a flipped sign of the
APIC affine term, a transposed C_p, a dropped gravity term, a wrong B-spline
branch, a flipped internal-force sign, F updated on the wrong side, ln J
replaced by J - 1, a wrong Drucker-Prager cone factor, a transposed APIC B_p,
a j-major block scan, and four mistakes in the P2G rounding scales that set
the GPU force tolerance (the particle volume without its 1/ppc, in both the
dense and the node-query scale; the stress term dropped; the APIC term of the
momentum scale dropped).  Each mutant is compiled to a temporary library and
the pin suite is run against it in a subprocess.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mpm_oracle.c")

MUTANTS = {
    "apic_sign": ("dmv[3 * q + r] = w[q] * mp * (v[r] + cd);", "dmv[3 * q + r] = w[q] * mp * (v[r] - cd);"),
    "apic_transposed_C": ("double cd = C[3 * r + 0] * d[0] + C[3 * r + 1] * d[1] + C[3 * r + 2] * d[2];",
                          "double cd = C[r + 0] * d[0] + C[r + 3] * d[1] + C[r + 6] * d[2];"),
    "no_gravity": ("vo[a] = vn + P->dt / m * (f[a] + m * P->g[a]);", "vo[a] = vn + P->dt / m * (f[a]);"),
    "bspline_center": ("*w = 0.75 - t * t;", "*w = 0.75 - 0.5 * t * t;"),
    "force_sign": ("df[3 * q + r] = -sg * Vp;", "df[3 * q + r] = sg * Vp;"),
    "F_right_multiply": ("matmul(G, F, Fn);", "matmul(F, G, Fn);"),
    "nh_J_minus_1": ("double lj = log(J);", "double lj = J - 1.0;"),
    "dp_factor": ("double dgamma = ndev + (3.0 * la + 2.0 * mu) / (2.0 * mu) * tr * alpha;",
                  "double dgamma = ndev + (3.0 * la + 2.0 * mu) / (3.0 * mu) * tr * alpha;"),
    "apic_B_transposed": ("Bm[3 * r + c] += w[q] * vn27[3 * q + r] * d[c];",
                          "Bm[3 * r + c] += w[q] * vn27[3 * q + c] * d[r];"),
    "abs_force_volume_no_ppc": ("af[3 * id + r] += g1 * particle_volume(P) * (tmax + mu + la);",
                                "af[3 * id + r] += g1 * P->h * P->h * P->h * (tmax + mu + la);"),
    "abs_force_no_stress": ("af[3 * id + r] += g1 * particle_volume(P) * (tmax + mu + la);",
                            "af[3 * id + r] += g1 * particle_volume(P) * (mu + la);"),
    "abs_momentum_no_C": ("s += fabs(C[9 * p + 3 * r + c]) * fabs(nodes[3 * q + c] * P->h - x[3 * p + c]);",
                          "s += 0.0;"),
    "node_scale_volume_no_ppc": ("af[k] += (fabs(gw[3 * q]) + fabs(gw[3 * q + 1]) + fabs(gw[3 * q + 2])) * particle_volume(P) *",
                                 "af[k] += (fabs(gw[3 * q]) + fabs(gw[3 * q + 1]) + fabs(gw[3 * q + 2])) * P->h * P->h * P->h *"),
    "scan_j_major": ("q = q * nb[ax] + (floordiv(n[ax], B) - blo[ax]);",
                     "q = q * nb[(ax + 1) % 3] + (floordiv(n[(ax + 1) % 3], B) - blo[(ax + 1) % 3]);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    with tempfile.TemporaryDirectory() as tmp:
        csrc = os.path.join(tmp, "mpm_oracle.c")
        open(csrc, "w").write(src.replace(old, new))
        open(os.path.join(tmp, "mpm_oracle.h"), "w").write(open(os.path.join(ROOT, "oracle", "mpm_oracle.h")).read())
        so = os.path.join(tmp, "libmut.so")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", so, csrc, "-lm"])
        env = dict(os.environ, MPM_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", "not sliding"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, "mutant %s survived every pin:\n%s" % (name, r.stdout[-2000:])
