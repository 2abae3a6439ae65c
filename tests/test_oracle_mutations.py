"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of ``oracle/fmm_oracle.cpp``:
a dropped term, a wrong sign, a wrong index or a swapped operand, in every stage
of the path (harmonics, P2M, M2M, M2L, L2L, L2P, P2P, keys, tree, MAC, the
particle-fitted centres and radii, traversal, adjoint, direct sum).  The copy is built with the oracle's own
compiler flags, and the pins of ``test_oracle_pins.py`` and the properties of
``test_oracle_properties.py`` run against it in a child process; at least one
must fail.  The unmutated copy goes through the
same harness and must pass, so that a broken harness cannot pass as a catch.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fmm_oracle.cpp")

# (name, anchor that opens the function, text to replace, replacement)
MUTANTS = [
    ("regular_seed_sign", "void regular(", "* (-xy) / (2.0 * m)", "* xy / (2.0 * m)"),
    ("regular_negative_m_phase", "void regular(",
     "U[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * std::conj(U[hidx(n, m)]);",
     "U[hidx(n, -m)] = std::conj(U[hidx(n, m)]);"),
    ("irregular_dropped_term", "void irregular(",
     "(2.0 * n - 1.0) * z * a - double((n + m - 1) * (n - m - 1)) * b) / r2",
     "(2.0 * n - 1.0) * z * a) / r2"),
    ("p2m_missing_conjugate", "void op_p2m(", "M[i] += q[j] * std::conj(U[i]);",
     "M[i] += q[j] * U[i];"),
    ("m2m_reversed_shift", "void op_m2m(",
     "double t[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};",
     "double t[3] = {cp[0] - cc[0], cp[1] - cc[1], cp[2] - cc[2]};"),
    ("m2m_dropped_degree", "void op_m2m(", "for (int k = 0; k <= n; ++k)",
     "for (int k = 0; k < n; ++k)"),
    ("m2l_sign", "void op_m2l(", "L[hidx(k, l)] += ((k & 1) ? -1.0 : 1.0) * s;",
     "L[hidx(k, l)] += s;"),
    ("m2l_order_index", "void op_m2l(", "T[hidx(n + k, m + l)]", "T[hidx(n + k, m - l)]"),
    ("m2l_reversed_distance", "void op_m2l(",
     "double d[3] = {cB[0] - cA[0], cB[1] - cA[1], cB[2] - cA[2]};",
     "double d[3] = {cA[0] - cB[0], cA[1] - cB[1], cA[2] - cB[2]};"),
    ("l2l_reversed_shift", "void op_l2l(",
     "double t[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};",
     "double t[3] = {cp[0] - cc[0], cp[1] - cc[1], cp[2] - cc[2]};"),
    ("l2l_order_index", "void op_l2l(", "int dl = l - i;", "int dl = i - l;"),
    ("l2p_dx_sign", "void op_l2p(", "cplx dxU = 0.5 * (up - um);", "cplx dxU = 0.5 * (up + um);"),
    ("l2p_dy_missing_i", "void op_l2p(", "cplx dyU = (up + um) / cplx(0.0, 2.0);",
     "cplx dyU = (up + um) / 2.0;"),
    ("keys_axes_swapped", "void root_and_keys(",
     "(spread3(k3[0]) << 2) | (spread3(k3[1]) << 1) | spread3(k3[2])",
     "(spread3(k3[2]) << 2) | (spread3(k3[1]) << 1) | spread3(k3[0])"),
    ("leaf_size_rule", "void build_cells(", "if (e - s <= t.ncrit) continue;",
     "if (e - s < t.ncrit) continue;"),
    ("tight_radius_not_max", "void tight_radii(", "best = std::max(best, d2);", "best = d2;"),
    ("tight_voxel_corner", "void tight_radii(", "const int64_t d = 2 * u[a] + 1 - ctr[a];",
     "const int64_t d = 2 * u[a] - ctr[a];"),
    ("fitted_centre_off_by_one", "void fitted_centres(",
     "ctr[a] = t.cint[3 * (size_t)c + a] = lo[a] + hi[a] + 1;",
     "ctr[a] = t.cint[3 * (size_t)c + a] = lo[a] + hi[a];"),
    ("fitted_radius_not_max", "void fitted_centres(", "best = std::max(best, d2);", "best = d2;"),
    ("fitted_mac_cube_distance", "bool mac(", "if (t.fitted) {", "if (false) {"),
    ("fitted_centre_unit", "void cell_centre(", "const double unit = std::ldexp(t.H, -MAXLEVEL);",
     "const double unit = std::ldexp(t.H, -MAXLEVEL + 1);"),
    ("mac_accepts_ties", "bool mac(", "return (t.theta * t.theta) * (double)D2 > (double)S2;",
     "return (t.theta * t.theta) * (double)D2 >= (double)S2;"),
    ("mac_theta_not_squared", "bool mac(",
     "return (t.theta * t.theta) * (double)D2 > (double)S2;",
     "return t.theta * (double)D2 > (double)S2;"),
    ("mac_circumscribed_factor", "bool mac(", "if (t.circumscribed) S2 *= 3;",
     "if (t.circumscribed) S2 *= 2;"),
    ("traversal_drops_child_self_pairs", "void visit(", "for (int j = i; j < t.nch[A]; ++j)",
     "for (int j = i + 1; j < t.nch[A]; ++j)"),
    ("traversal_one_way_m2l", "void visit(",
     "m2l.push_back({B, A});\n      m2l.push_back({A, B});", "m2l.push_back({B, A});"),
    ("centre_at_corner", "void cell_centre(",
     "out[0] = t.r0[0] + (2.0 * t.ix[c] + 1.0) * R;", "out[0] = t.r0[0] + (2.0 * t.ix[c]) * R;"),
    ("l2l_skips_deepest_level", "// downward pass: L2L top down",
     "for (int l = 1; l < nlev; ++l) {", "for (int l = 1; l < nlev - 1; ++l) {"),
    ("p2p_gradient_sign", "void evaluate(", "g[0] -= f * dx;", "g[0] += f * dx;"),
    ("p2p_drops_last_source", "void evaluate(",
     "for (int j = t.bbeg[a]; j < t.bend[a]; ++j) {",
     "for (int j = t.bbeg[a]; j < t.bend[a] - 1; ++j) {"),
    ("adjoint_dropped_term", "int orc_backward(",
     "dx[3 * i + a] = w[i] * gq[3 * i + a] + qq[i] * gw[3 * i + a];",
     "dx[3 * i + a] = w[i] * gq[3 * i + a];"),
    ("direct_gradient_sign", "int orc_direct(", "g0 -= f * dx;", "g0 += f * dx;"),
]

RUNNER = (
    "import sys, oracle, pytest\n"
    "oracle.use_library(sys.argv[1])\n"
    "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu',\n"
    "                      'tests/test_oracle_pins.py', 'tests/test_oracle_properties.py']))\n"
)


def mutate(src: str, anchor: str, old: str, new: str) -> str:
    assert src.count(anchor) == 1, f"anchor {anchor!r} not unique"
    i = src.index(anchor)
    j = src.find(old, i)
    assert j >= 0, f"{old!r} not found after {anchor!r}"
    return src[:j] + new + src[j + len(old):]


def _run_pins(so: str) -> int:
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-c", RUNNER, so], cwd=ROOT, env=env,
                       stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL, timeout=600)
    return r.returncode


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_every_planted_mistake_fails_a_pin(tmp_path):
    import oracle
    src = open(SRC).read()
    cases = [("unmutated", src)] + [(n, mutate(src, a, o, w)) for n, a, o, w in MUTANTS]
    names = [n for n, _ in cases]
    assert len(set(names)) == len(names)

    def build(case):
        name, text = case
        cpp = tmp_path / f"{name}.cpp"
        cpp.write_text(text)
        so = str(tmp_path / f"lib{name}.so")
        oracle.compile_library(str(cpp), so)
        return so

    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        libs = list(ex.map(build, cases))
    with ThreadPoolExecutor(max(1, workers // 2)) as ex:
        codes = dict(zip(names, ex.map(_run_pins, libs)))
    assert codes["unmutated"] == 0, "the harness fails the unmutated oracle"
    survivors = [n for n in names[1:] if codes[n] == 0]
    assert not survivors, f"mistakes no pin catches: {survivors}"
