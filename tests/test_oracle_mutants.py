"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that the pins
of test_oracle_pins.py catch every one: a dropped term, a wrong sign or index, a transposed
operand, a wrong scale.  Each mutant is compiled from a patched copy of fdtd_oracle.c and
the pins run against it in a subprocess."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fdtd_oracle.c")

# (name, original text, mutated text); each original must occur in the source
MUTANTS = [
    ("h_update_sign", "Hx[c] = old - Ch * (D / ay.kH[j] + pHx[c]);",
     "Hx[c] = old + Ch * (D / ay.kH[j] + pHx[c]);"),
    ("h_cpml_term_dropped", "Hy[c] = old + Ch * (D / ax.kH[i] + pHy[c]);",
     "Hy[c] = old + Ch * (D / ax.kH[i]);"),
    ("e_stencil_index", "double Dx = (Hy[c] - Hy[c - 1]) / dx;\n                double Dy = (Hx[c] - Hx[c - nx]) / dy;\n                pEx[c]",
     "double Dx = (Hy[c + 1] - Hy[c]) / dx;\n                double Dy = (Hx[c] - Hx[c - nx]) / dy;\n                pEx[c]"),
    ("loss_half_dropped", "double EA = OR_EPS0 * eps_r[c] / g->dt + 0.5 * sigma[c];",
     "double EA = OR_EPS0 * eps_r[c] / g->dt + sigma[c];"),
    ("source_scale", "Q[c] -= wav[(size_t)s * nt + n] / (dx * dy);\n        }\n        for (int j = 1; j <= ny - 2; ++j)\n            for (int i = 1; i <= nx - 2; ++i) {\n                size_t c = (size_t)j * nx + i;\n                Ez[c] = Ca[c]",
     "Q[c] -= wav[(size_t)s * nt + n] / dx;\n        }\n        for (int j = 1; j <= ny - 2; ++j)\n            for (int i = 1; i <= nx - 2; ++i) {\n                size_t c = (size_t)j * nx + i;\n                Ez[c] = Ca[c]"),
    ("adjoint_transposed_index", "aHy[c - 1] -= aDx / dx;", "aHy[c + 1] -= aDx / dx;"),
    ("adjoint_ca_dropped", "aEz[c] = Ca[c] * aEz[c];", "aEz[c] = aEz[c];"),
    ("gradient_sign", "if (g_sigma) g_sigma[c] += -lam * 0.5 * (E1[c] + E0[c]);",
     "if (g_sigma) g_sigma[c] += lam * 0.5 * (E1[c] + E0[c]);"),
    ("adjoint_cpml_decay_dropped", "aPHx[c] *= ay.bH[j];", "(void)0;"),
    ("receiver_after_update", "traces[(size_t)n * nrec + r] = Ez[(size_t)rec[2 * r + 1] * nx + rec[2 * r]];",
     "traces[(size_t)n * nrec + r] = n > 0 ? ez_hist_unused_guard(Ez, rec, r, nx) : 0.0;"),
]

# mistakes in the TE-mode forward model, caught by the pins of test_oracle_te_pins.py
TE_MUTANTS = [
    ("te_hz_update_sign", "Hz[c] = old + Ch * (Dy / ay.kH[j]", "Hz[c] = old - Ch * (Dy / ay.kH[j]"),
    ("te_hz_cpml_term_dropped", "- Dx / ax.kH[i] - pHzx[c]);", "- Dx / ax.kH[i]);"),
    ("te_ex_stencil_index", "double D = (Hz[c] - Hz[c - nx]) / dy;",
     "double D = (Hz[c + nx] - Hz[c]) / dy;"),
    ("te_ey_sign", "Qy[c] = -(D / ax.kE[i] + pEyx[c]);", "Qy[c] = (D / ax.kE[i] + pEyx[c]);"),
    ("te_source_component", "double* Q = pol == 0 ? Qx : Qy;", "double* Q = pol == 0 ? Qy : Qx;"),
    ("te_coefficient_cell", "Ex[c] = Ca[c] * Ex[c] + Cb[c] * Qx[c];",
     "Ex[c] = Ca[c + 1] * Ex[c] + Cb[c + 1] * Qx[c];"),
    ("te_receiver_node", "traces[((size_t)n * nrec + r) * 3 + 0] = Ex[c];",
     "traces[((size_t)n * nrec + r) * 3 + 0] = Ex[c + 1];"),
    ("te_source_scale", "Qy;\n            Q[c] -= wav[(size_t)s * nt + n] / (dx * dy);",
     "Qy;\n            Q[c] -= wav[(size_t)s * nt + n] / dx;"),
    ("te_hz_receiver_node", "traces[((size_t)n * nrec + r) * 3 + 2] = Hz[c];",
     "traces[((size_t)n * nrec + r) * 3 + 2] = Hz[c + nx];"),
    # ... and in its adjoint
    ("te_adj_psi_decay_dropped", "aPHzx[c] = ax.bH[i] * aPHzx[c] - ah;", "aPHzx[c] = -ah;"),
    ("te_adj_transposed_index", "aHz[c - 1] -= aD / dx;", "aHz[c + 1] -= aD / dx;"),
    ("te_adj_gradient_sign", "if (g_sigma) g_sigma[c] += -lam * 0.5 * (Y1[c] + Y0[c]);",
     "if (g_sigma) g_sigma[c] += lam * 0.5 * (Y1[c] + Y0[c]);"),
    ("te_adj_ca_dropped", "aEx[c] = Ca[c] * ae;", "aEx[c] = ae;"),
    ("te_adj_receiver_component", "double* aE = pol == 0 ? aEx : aEy;",
     "double* aE = pol == 0 ? aEy : aEx;"),
]

PREAMBLE = "static double ez_hist_unused_guard(const double* E, const int32_t* rec, int r, int nx) { return 2.0 * E[(size_t)rec[2 * r + 1] * nx + rec[2 * r]]; }\n"

PINS = ("energy or reciprocity or dot_product or analytic or zero_lag or fd_every_cell "
        "or tangent_linear or wavelet_gradient or cpml_reflection")


def _run_mutant(tmp, name, a, b, pins_file="test_oracle_pins.py", pins=PINS):
    src = open(SRC).read()
    assert a in src, name
    mutated = src.replace("#define OR_MU0", PREAMBLE + "#define OR_MU0", 1).replace(a, b, 1)
    path = os.path.join(tmp, f"{name}.c")
    with open(path, "w") as f:
        f.write(mutated)
    lib = O.build(src=path, out=os.path.join(tmp, f"lib{name}.so"))
    env = dict(os.environ, GPRFWI_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins_file), "-k", pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    last = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    # caught = a pin assertion failed (not an import, collection or build error)
    caught = r.returncode == 1 and " failed" in last and "error" not in last
    return name, caught, last


def test_every_planted_mistake_fails_a_pin(tmp_path):
    te = [m + ("test_oracle_te_pins.py", "te_") for m in TE_MUTANTS]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda m: _run_mutant(str(tmp_path), *m), MUTANTS + te))
    survivors = [(n, last) for n, caught, last in results if not caught]
    assert not survivors, f"mutants not caught by any pin: {survivors}"
