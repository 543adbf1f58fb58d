"""The oracle's pins are sensitive: each plausible mistake below, planted in a
copy of the oracle's C source and built on the CPU, makes the pin suite fail.

Each mutation names the pin expected to catch it; the test only requires that
the selected pin files fail as a whole."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hsg_oracle.c")

MUTATIONS = {
    # field: J instead of J^T on the backward bond (local gauge, gradient)
    "field_transpose": ("h[a] += Jdn[mu * 9 + b * 3 + a] * s_dn[mu * 3 + b];",
                        "h[a] += Jdn[mu * 9 + a * 3 + b] * s_dn[mu * 3 + b];",
                        ["test_oracle_updates.py"]),
    # heat-bath: density exp(kappa u / 2) instead of exp(kappa u)
    "hb_half_kappa": ("w = -log1p(r0 * expm1(-2.0 * kappa)) / kappa;",
                      "w = -log1p(r0 * expm1(-kappa)) / kappa;",
                      ["test_oracle_updates.py"]),
    # heat-bath: kappa from |h|^2
    "hb_kappa_hh": ("double kappa = beta * hn;", "double kappa = beta * hh;",
                    ["test_oracle_updates.py"]),
    # frame: wrong sign in e2 (not orthonormal)
    "frame_sign": ("double e2[3] = {q, sgn + n[1] * n[1] * p, -n[1]};",
                   "double e2[3] = {q, sgn + n[1] * n[1] * p, n[1]};",
                   ["test_oracle_updates.py"]),
    # overrelaxation: projection instead of reflection
    "or_projection": ("double f = 2.0 * hs / hh;", "double f = hs / hh;",
                      ["test_oracle_updates.py"]),
    # energy counts the bond to the backward neighbour too
    "energy_double": ("long up = neighbour(L, i, mu, +1);\n      const double *J = J9",
                      "long up = neighbour(L, i, mu, -1);\n      const double *J = J9",
                      ["test_oracle_updates.py", "test_oracle_pt_measure.py"]),
    # PT: Metropolis exponent with the wrong sign
    "pt_sign": ("double delta = (beta[i] - beta[i + 1]) * (E[a] - E[b]);",
                "double delta = (beta[i + 1] - beta[i]) * (E[a] - E[b]);",
                ["test_oracle_pt_measure.py"]),
    # chirality: backward neighbour taken along the next axis
    "chirality_nbr": ("long dn = neighbour(L, i, mu, -1);\n  const double *a",
                      "long dn = neighbour(L, i, (mu + 1) % 3, -1);\n  const double *a",
                      ["test_oracle_pt_measure.py"]),
    # Fourier phase with the wrong sign convention
    "fourier_sign": ("double cr = cos(ph), ci = sin(ph);", "double cr = cos(ph), ci = -sin(ph);",
                     ["test_oracle_pt_measure.py"]),
    # Philox: a dropped key bump
    "philox_keybump": ("      k1 = (k1 + W1) & mask;\n", "",
                       ["test_oracle_philox.py"]),
    # Philox: high and low halves of one product exchanged
    "philox_hilo": ("uint64_t n1 = lo1;", "uint64_t n1 = hi1;",
                    ["test_oracle_philox.py"]),
    # sweep: the black half applied twice, the white half never
    "sweep_colours": ("  oracle_half_sweep(L, J9, s, 1, kind, beta, seed, lattice, t);\n}",
                      "  oracle_half_sweep(L, J9, s, 0, kind, beta, seed, lattice, t);\n}",
                      ["test_oracle_updates.py"]),
    # sequential overrelaxation: sites visited in reverse order
    "sequential_reverse": ("  for (long i = 0; i < N; ++i) {\n    double h[3], s_new[3];\n    oracle_local_field(L, J9, s, i, h);\n    oracle_or_update(h, s + i * 3, s_new);",
                           "  for (long i = N - 1; i >= 0; --i) {\n    double h[3], s_new[3];\n    oracle_local_field(L, J9, s, i, h);\n    oracle_or_update(h, s + i * 3, s_new);",
                           ["test_oracle_sequential.py"]),
    # bimodal couplings: D^xz and D^yz bits exchanged
    "bimodal_bit_order": ("M[0] = iso + d[0]; M[1] = d[3];       M[2] = d[4];",
                          "M[0] = iso + d[0]; M[1] = d[3];       M[2] = d[5];",
                          ["test_oracle_bimodal.py"]),
    # bimodal couplings: the isotropic sign also added off the diagonal
    "bimodal_iso_offdiag": ("M[3] = d[3];       M[4] = iso + d[1]; M[5] = d[5];",
                            "M[3] = iso + d[3]; M[4] = iso + d[1]; M[5] = d[5];",
                            ["test_oracle_bimodal.py"]),
    # field: one component with the wrong sign on white sites only
    "white_field_sign": ("    if (site_colour(L, i) != colour) continue;\n    double h[3], s_new[3];\n    oracle_local_field(L, J9, s, i, h);",
                      "    if (site_colour(L, i) != colour) continue;\n    double h[3], s_new[3];\n    oracle_local_field(L, J9, s, i, h);\n    if (colour == 1) { h[0] = -h[0]; }",
                      ["test_oracle_updates.py"]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new, files = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut = src.replace(old, new)
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(mut)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-D_GNU_SOURCE", str(c), "-o", str(so), "-lm"],
                   check=True)
    env = dict(os.environ, HSG_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                       + [os.path.join(ROOT, "tests", f) for f in files],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"
