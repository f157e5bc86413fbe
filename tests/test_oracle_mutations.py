"""The oracle's pins catch plausible misreadings of the paper.

Each case below alters one constant or operation of the oracle's source the way a misreading of
the paper would -- an exponent of eq. 19 / Alg. 1 or of the CTENOZ measure of Alg. 2, the average
over s_t - 1 directional stencils, the "1 +" of the CTENOZ weight, the cut-off C_T of eq. 23, the
linear coefficients of eq. 18, the CWENO exponent of eq. 14, the division by lambda_1 in eq. 17,
the smoothness integral of eq. 15, the Roe averages, wave speeds and star states of eqs. 25-29,
the SSP-RK3 and RK4 weights, the reflected wall state, the transmissive and moving-shock boundary
states, the face quadrature and area weights, the characteristic eigenvectors, the sum over faces
of the CFL step -- compiles the altered copy, and runs the pins that
should notice against it: at least one of them must fail. An unaltered copy compiled the same way
must pass all of them, which shows that the altered build is the one under test.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cteno_oracle.c")
SELECTION = (os.path.join(ROOT, "tests", "test_oracle_selection_pins.py"), None)
HLLC = (os.path.join(ROOT, "tests", "test_oracle_pins.py"), "hllc")
WALLS = (os.path.join(ROOT, "tests", "test_oracle_walls_rk4.py"), "walls_conserve or flow_into_a_wall")
RK4 = (os.path.join(ROOT, "tests", "test_oracle_walls_rk4.py"), "runge_kutta_order or rk4_step")
CHAR = (os.path.join(ROOT, "tests", "test_oracle_characteristic.py"), "eigenvectors or smooth_field or contact")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, text in the oracle, misread replacement[, pins: (file, -k expression)]); the text occurs
# once, except where noted; the pins default to the selection and time-step pins
MUTATIONS = [
    ("CTENO gamma exponent 6 -> 4",
     "gam[s] = 1.0 / pow(SI[s] + p->eps, 6.0);", "gam[s] = 1.0 / pow(SI[s] + p->eps, 4.0);"),
    ("CTENOZ tau exponent 6 -> 2",
     "if (p->ctenoz_form == 0) tau = pow(tau, 6.0);", "if (p->ctenoz_form == 0) tau = pow(tau, 2.0);"),
    ("tau averaged over s_t instead of s_t - 1",
     "tau = acc / (st - 1);", "tau = acc / st;"),
    ("'1 +' dropped from the CTENOZ weight",
     "if (p->ctenoz_form == 0) gam[s] = 1.0 + tau / (SI[s] + p->eps);",
     "if (p->ctenoz_form == 0) gam[s] = tau / (SI[s] + p->eps);"),
    ("cut-off 10 C_T",
     "if (!(chi[s] < p->C_T)) bits |= 1u << s;", "if (!(chi[s] < 10.0 * p->C_T)) bits |= 1u << s;"),
    ("lambda_s over s_t instead of s_t - 1 (in the selection and in p_1 of eq. 17: both places)",
     "const double lams = (st > 1) ? (1.0 - lam1) / (st - 1) : 0.0;",
     "const double lams = (st > 1) ? (1.0 - lam1) / st : 0.0;"),
    ("WENO-Z form power 6 -> 4",
     "else gam[s] = 1.0 + pow(tau / (SI[s] + p->eps), 6.0);",
     "else gam[s] = 1.0 + pow(tau / (SI[s] + p->eps), 4.0);"),
    ("CWENO exponent 4 -> 2",
     "gam[s] = ((s == 0) ? lam1 : lams) / pow(p->eps + SI[s], 4.0);",
     "gam[s] = ((s == 0) ? lam1 : lams) / pow(p->eps + SI[s], 2.0);"),
    ("time step with the largest face term instead of the sum over faces",
     "s += o->area[i * nf + f] * (fabs(un) + c);", "s = fmax(s, o->area[i * nf + f] * (fabs(un) + c));"),
    ("p_1 without the division by lambda_1 (eq. 17)",
     "a1[k] = s / lam1;", "a1[k] = s;", (HLLC[0], "eq17")),
    ("smoothness indicator not scaled by the reference volume |V0'| (eq. 15)",
     "si += v0 * s;", "si += s;", (HLLC[0], "smoothness")),
    ("smoothness indicator from the first derivatives only (eq. 15)",
     "if (na > deg) continue;", "if (na > deg || na > 1) continue;", (HLLC[0], "smoothness")),
    ("Roe average weighted by rho_R / rho_L instead of its square root (eq. 26)",
     "double D = sqrt(rR / rL);", "double D = rR / rL;", HLLC),
    ("Roe enthalpy as the arithmetic mean (eq. 26)",
     "double Ht = (HL + HR * D) / (1.0 + D);", "double Ht = 0.5 * (HL + HR);", HLLC),
    ("S_R without the Roe-averaged speed (eq. 25)",
     "SR = fmax(unR + cR, utn + ct)", "SR = (unR + cR)", HLLC),
    ("SSP-RK3 second stage with weights 1/2, 1/2",
     "a[3] = {0.0, 0.75, 1.0 / 3.0}, b[3] = {1.0, 0.25, 2.0 / 3.0}",
     "a[3] = {0.0, 0.5, 1.0 / 3.0}, b[3] = {1.0, 0.5, 2.0 / 3.0}", (HLLC[0], "ssp_rk3")),
    ("HLLC star momentum with p* + p_L (eq. 29)",
     "us[1 + j] = ((SL - unL) * uL[1 + j] + (ps - pL) * n[j]) * f;",
     "us[1 + j] = ((SL - unL) * uL[1 + j] + (ps + pL) * n[j]) * f;", HLLC),
    ("HLLC star energy without the p_L u_L term (eq. 29)",
     "us[d + 1] = ((SL - unL) * uL[d + 1] - pL * unL + ps * SM) * f;",
     "us[d + 1] = ((SL - unL) * uL[d + 1] + ps * SM) * f;", HLLC),
    ("wall state with the normal momentum subtracted once instead of reflected",
     "ub[1 + k] = uL[1 + k] - 2.0 * mn * n[k];", "ub[1 + k] = uL[1 + k] - mn * n[k];", WALLS),
    ("RK4 last stage with dt/3",
     "o->U[k] = o->Acc[k] + dk / 6.0;", "o->U[k] = o->Acc[k] + dk / 3.0;", RK4),
    ("RK4 second stage accumulated with dt/6",
     "o->Acc[k] += dk / 3.0;\n        o->U[k] = o->Un[k] + 0.5 * dk;",
     "o->Acc[k] += dk / 6.0;\n        o->U[k] = o->Un[k] + 0.5 * dk;", RK4),
    ("left eigenvector of u_n - c with the sign of u_n / c flipped",
     "L[0][0] = 0.5 * (b2 + un / c);", "L[0][0] = 0.5 * (b2 - un / c);", CHAR),
    ("left eigenvector of u_n - c with the sign of n / c flipped",
     "L[0][1 + j] = 0.5 * (-b1 * vel[j] - n[j] / c);", "L[0][1 + j] = 0.5 * (-b1 * vel[j] + n[j] / c);", CHAR),
    ("least-squares rows without the member volumes |V'_m| (eq. 10, reading R6)",
     "for (int k = 0; k < c->nst; ++k) b[k] = c->Vp[k] * (U[v * n + c->ids[k]] - U0[v]); /* eq. 10 */",
     "for (int k = 0; k < c->nst; ++k) b[k] = (U[v * n + c->ids[k]] - U0[v]); /* eq. 10 */",
     (PINS, "linear_fields_reproduced")),
    ("characteristic face values transformed back with L^T instead of R",
     "for (int w = 0; w < nv; ++w) s += R[v][w] * W[q][w];",
     "for (int w = 0; w < nv; ++w) s += L[w][v] * W[q][w];", CHAR),
    ("characteristic mean of field w taken as the conserved mean of variable w",
     "for (int v = 0; v < nv; ++v) Wbar += L[w][v] * U0[v];", "Wbar = U0[w];", CHAR),
    ("transmissive outside state the reconstructed inside value instead of the cell mean",
     "for (int v = 0; v < nv; ++v) ub[v] = o->U[v * o->ncells + i];",
     "for (int v = 0; v < nv; ++v) ub[v] = uL[v];", (PINS, "transmissive_inflow")),
    ("moving-shock boundary without the shock's motion",
     "use_a = o->shock[0] + o->shock[1] * mid[1] + o->shock[2] * o->stage_time > mid[0];",
     "use_a = o->shock[0] + o->shock[1] * mid[1] > mid[0];",
     (os.path.join(ROOT, "tests", "test_oracle_walls_rk4.py"), "moving_shock")),
    ("face flux not weighted by the face area (eq. 2)",
     "acc[v] += o->fw[q] * o->area[i * nf + f] * F[v];", "acc[v] += o->fw[q] * F[v];",
     (PINS, "free_stream or conservation")),
    ("edge Gauss points moved (2D face rule)",
     "t[0][0] = 0.5 * (1.0 - g); /* fraction", "t[0][0] = 0.5 * (1.0 - 0.9 * g); /* fraction", (PINS, "face_rule")),
    ("Gauss-Jacobi weight of the 3D face rule",
     "double wu2 = (1.0 / 6.0 - 0.5 * u[0]) / (u[1] - u[0]);",
     "double wu2 = (1.0 / 6.0 - 0.4 * u[0]) / (u[1] - u[0]);", (PINS, "face_rule")),
]


def _compile(src_text: str, out: str) -> None:
    path = out[:-3] + ".c"
    with open(path, "w") as f:
        f.write(src_text)
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", path, "-o", out, "-lm"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            return
    raise RuntimeError("oracle copy did not compile:\n" + r.stderr)


def _run_pins(lib: str, pins) -> tuple[int, int]:
    """Run the pins against the given oracle build; (return code, number of failed pins)."""
    env = dict(os.environ, CTENO_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    path, expr = pins
    cmd = [sys.executable, "-m", "pytest", path, "-q", "-p", "no:cacheprovider"] + (["-k", expr] if expr else [])
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True)
    m = re.search(r"(\d+) failed", r.stdout)
    return r.returncode, int(m.group(1)) if m else 0


def test_every_misreading_fails_a_pin():
    with open(SRC) as f:
        source = f.read()
    for name, old, *_ in MUTATIONS:
        want = 2 if name.startswith("lambda_s") else 1
        assert source.count(old) == want, f"{name}: the oracle no longer holds {old!r} {want} time(s)"
    pin_sets = sorted({tuple(m[3]) if len(m) > 3 else SELECTION for m in MUTATIONS}, key=str)
    jobs = [(f"unaltered ({os.path.basename(p)} {k or ''})", source, (p, k)) for p, k in pin_sets]
    jobs += [(m[0], source.replace(m[1], m[2]), m[3] if len(m) > 3 else SELECTION) for m in MUTATIONS]
    with tempfile.TemporaryDirectory() as tmp:
        def one(k):
            name, text, pins = jobs[k]
            lib = os.path.join(tmp, f"orc{k}.so")
            _compile(text, lib)
            return name, _run_pins(lib, pins)

        with cf.ThreadPoolExecutor(max_workers=4) as ex:
            results = list(ex.map(one, range(len(jobs))))
    nc = len(pin_sets)
    for name, control in results[:nc]:
        assert control == (0, 0), f"the {name} copy fails its pins: {control}"
    altered = results[nc:]
    caught = {name: nfail for name, (rc, nfail) in altered}
    # a case counts as caught only when pins ran and failed (not on a crash or a collection error)
    missed = [name for name, (rc, nfail) in altered if not (rc == 1 and nfail > 0)]
    assert not missed, f"misreadings no pin catches: {missed} (failed pins per case: {caught})"
    print("failed pins per misreading:", caught)


if __name__ == "__main__":
    pytest.main([__file__, "-q", "-s"])
