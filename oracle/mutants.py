"""Planted mistakes for the pin-strength tests.

TEST INFRASTRUCTURE ONLY.  Each entry turns one exact snippet of ``rod_oracle.c`` into a
plausible mistake (a dropped term, a flipped sign, a transposed operand, a wrong factor or
index).  ``build_mutant(mid)`` writes a patched copy of the source with that one change and
compiles it into a library of its own, so the oracle that the other tests use carries no
switch and no trace of the mistakes.  Every snippet must occur exactly once in the source.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_OUT = os.path.join(_ROOT, "_build", "oracle_mutants")

# id: (description, snippet of rod_oracle.c, replacement)
MUTANTS = {
    1: ("bending couple without the (kappa x m) averaging term",
        "tot[c] = (Pi - Pm) + 0.5 * (Tm + Ti) + tau[c * E + ie];",
        "tot[c] = (Pi - Pm) + tau[c * E + ie];"),
    2: ("shear couple with the wrong sign",
        "tau[c * E + ie] = ts[c] * rl + tl[c] + Jw[c] / (e * e) * edot;",
        "tau[c * E + ie] = -ts[c] * rl + tl[c] + Jw[c] / (e * e) * edot;"),
    3: ("internal force without the 1/e factor",
        "for (int c = 0; c < 3; ++c) Nl[c] = Nl[c] / e;",
        "/* no 1/e */"),
    4: ("shear strain from Q^T l instead of Q l",
        "double tt[3] = {l[0] / lg, l[1] / lg, l[2] / lg};\n      mat_vec(M, l, Ql);",
        "double tt[3] = {l[0] / lg, l[1] / lg, l[2] / lg};\n      matT_vec(M, l, Ql);"),
    5: ("angular balance without the (J w/e^2) de/dt term",
        "tau[c * E + ie] = ts[c] * rl + tl[c] + Jw[c] / (e * e) * edot;",
        "tau[c * E + ie] = ts[c] * rl + tl[c];"),
    6: ("angular balance without the (J w/e) x w term",
        "tau[c * E + ie] = ts[c] * rl + tl[c] + Jw[c] / (e * e) * edot;",
        "tau[c * E + ie] = ts[c] * rl + Jw[c] / (e * e) * edot;"),
    7: ("director update exp(+h[w]x) instead of exp(-h[w]x)",
        "phi[c] = -h * w[c * E + i];",
        "phi[c] = h * w[c * E + i];"),
    8: ("bending couple divided by eps^2 instead of eps^3",
        "double eps3 = eps * eps * eps;",
        "double eps3 = eps * eps;"),
    9: ("curvature from +log instead of -log",
        "kap[c] = -phi[c] / D;",
        "kap[c] = phi[c] / D;"),
    10: ("contact force split (s, 1-s) instead of (1-s, s)",
         "double wa = 1.0 - s;",
         "double wa = s;"),
    11: ("dashpot with the wrong sign",
         "fmag = fmag - p->contact_c * dot3(vrel, nrm);",
         "fmag = fmag + p->contact_c * dot3(vrel, nrm);"),
    12: ("cell list missing the -x neighbour cells",
         "for (int dx = -1; dx <= 1 && !stop; ++dx) {",
         "for (int dx = 0; dx <= 1 && !stop; ++dx) {"),
    14: ("node mass doubled",
         "double mass = 0.5 * K.rho * K.A * (rl_l + rl_r);\n      double rlN",
         "double mass = 1.0 * K.rho * K.A * (rl_l + rl_r);\n      double rlN"),
    15: ("no rotational damping",
         "tot[c] += -p->nu_damp * rl * (K.I[c] / K.A) * wi[c];",
         "/* no rotational damping */"),
    17: ("angular acceleration without the e factor",
         "acc_w[c * E + ie] = dil[ie] * tot[c] / (K.rho * rl * K.I[c]);",
         "acc_w[c * E + ie] = tot[c] / (K.rho * rl * K.I[c]);"),
    19: ("gravity with the wrong sign",
         "F[c] += mass * p->gravity[c];",
         "F[c] -= mass * p->gravity[c];"),
    20: ("actuation couple on the clamped element",
         "return (clamped && p->n_elem[r] >= 2) ? 1 : 0;",
         "return 0 * clamped;"),
    21: ("no Stokes drag",
         "F[c] += -(p->nu_damp + p->stokes_gamma) * rlN * vj[c];",
         "F[c] += -p->nu_damp * rlN * vj[c];"),
    22: ("magnetic couple with Q^T b instead of Q b",
         "qb[a] = M[3 * a] * bt[0] + M[3 * a + 1] * bt[1] + M[3 * a + 2] * bt[2];",
         "qb[a] = M[a] * bt[0] + M[3 + a] * bt[1] + M[6 + a] * bt[2];"),
    23: ("muscle couples tau_i - tau_{i-1} instead of tau_{i-1} - tau_i",
         "tot[0] += tl - tr;",
         "tot[0] += tr - tl;"),
    24: ("wall contact without the rod radius",
         "double delta = p->radius[r] - dot3(d, nn);",
         "double delta = 0.0 - dot3(d, nn);"),
    25: ("friction along the sliding direction instead of against it",
         "(mu > 0.0 && fn > 0.0) ? -mu * fn * vt[c] / den : 0.0;",
         "(mu > 0.0 && fn > 0.0) ? mu * fn * vt[c] / den : 0.0;"),
    26: ("energy: bend/twist term over one element's rest length instead of the Voronoi length",
         "double D = 0.5 * (p->rest_len[g.elem0 + k] + p->rest_len[g.elem0 + k + 1]);",
         "double D = p->rest_len[g.elem0 + k];"),
    27: ("energy: rotational kinetic term with I_1 about every axis",
         "H += 0.5 * K.rho * rl * K.I[c] * wc * wc;",
         "H += 0.5 * K.rho * rl * K.I[0] * wc * wc;"),
    28: ("energy: shear terms with the axial stiffness E A",
         "H += 0.5 * rl * K.S[c] * sc * sc;",
         "H += 0.5 * rl * K.S[2] * sc * sc;"),
    29: ("energy: work potential of gravity with the wrong sign",
         "H -= mass * dot3(p->gravity, xj);",
         "H += mass * dot3(p->gravity, xj);"),
    30: ("energy: translational kinetic term without the 1/2",
         "H += 0.5 * mass * dot3(vj, vj);",
         "H += 1.0 * mass * dot3(vj, vj);"),
}


def mutant_source(mid: int) -> str:
    """rod_oracle.c with mistake `mid` planted (its snippet must occur exactly once)."""
    with open(os.path.join(_HERE, "rod_oracle.c")) as f:
        src = f.read()
    _, old, new = MUTANTS[mid]
    n = src.count(old)
    if n != 1:
        raise RuntimeError(f"mutant {mid}: snippet found {n} times in rod_oracle.c")
    return src.replace(old, new)


def build_mutant(mid: int) -> str:
    """Compile the oracle with mistake `mid` into its own shared library; returns its path."""
    os.makedirs(_OUT, exist_ok=True)
    src = os.path.join(_OUT, f"rod_oracle_m{mid}.c")
    lib = os.path.join(_OUT, f"liboracle_m{mid}.so")
    text = mutant_source(mid)
    base = os.path.join(_HERE, "rod_oracle.c")
    deps = [base, os.path.join(_HERE, "rod_oracle.h"), os.path.abspath(__file__)]
    if os.path.exists(lib) and all(os.path.getmtime(lib) >= os.path.getmtime(d) for d in deps):
        return lib
    with open(src, "w") as f:
        f.write(text)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas",
                    "-I", _HERE, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib
