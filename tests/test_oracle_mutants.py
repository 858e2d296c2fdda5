"""Planted mistakes: every pin of the oracle is worth something only if a
plausible error in the oracle makes one of them fail. Each case below
copies the oracle's source, plants one mistake by a one-line textual edit
(a wrong sign, a swapped operand, an inclusive bin edge, ...), compiles the
copy into a temporary library, and runs the CPU pin suites against it in a
child process (the oracle loader takes the library from GS_ORACLE_LIB).
The test passes only when the pins fail for every planted mistake; the
unmodified source must pass the same suites (checked first)."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gs_oracle.cpp")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_rounding.py",
        "tests/test_oracle_tooling.py", "tests/test_oracle_connected.py",
        "tests/test_oracle_pixel.py", "tests/test_oracle_mu.py"]

# (name, text in the oracle, replacement)
MUTANTS = [
    ("sign of the parity volume", "if (V != 0) s = V > 0 ? 1 : -1;", "if (V != 0) s = V > 0 ? -1 : 1;"),
    ("swapped edge-bin slots of a tetrahedron",
     "Tup6 t = {g.bin[p1], g.bin[p2], g.bin[al], g.bin[q12], g.bin[be], g.bin[ga]};",
     "Tup6 t = {g.bin[p1], g.bin[p2], g.bin[al], g.bin[be], g.bin[q12], g.bin[ga]};"),
    ("inclusive outer bin edge", "D2 >= g.edges2[g.nb]) return -1;", "D2 > g.edges2[g.nb]) return -1;"),
    ("inner bin edge on the wrong side", "g.edges2[b + 1] <= D2) ++b;", "g.edges2[b + 1] < D2) ++b;"),
    ("minimum image that never wraps negative displacements", "else if (2 * d < -box) d += box;",
     "else if (d < -box) d += box;"),
    ("wrong pairing in the disconnected term",
     "      volatile double t2 = x[r[1]] * x[r[4]];", "      volatile double t2 = x[r[1]] * x[r[3]];"),
    ("chirality from even instead of odd permutations",
     "if (perms[q].sign < 0 && relabel", "if (perms[q].sign > 0 && relabel"),
    ("round half up instead of to even", "if (half && (rest || (q & 1ull))) q += 1;",
     "if (half) q += 1;"),
    ("third triangle side read from the hub row",
     "const int c = conf.of(b_ij, g.bin[a], g.bin[b]);", "const int c = conf.of(b_ij, g.bin[a], g.bin[a]);"),
    ("a weight factor repeated", "(i128)fw.W[i] * fw.W[j] * fw.W[ka]", "(i128)fw.W[i] * fw.W[j] * fw.W[j]"),
    ("lattice rounding instead of flooring", "(int64_t)std::floor(pos[i] * 1024.0)",
     "(int64_t)std::round(pos[i] * 1024.0)"),
    ("pixel sector edge on the diagonal on the wrong side", "if (b >= a) ++sub;",
     "if (b > a) ++sub;"),
    ("pixel bands shifted by one edge", "if (z_at_least(z, n2, k - 8)) ++band;",
     "if (z_at_least(z, n2, k - 7)) ++band;"),
    ("pixel parity without the relabelling sign",
     "s = (Vp > 0 ? 1 : -1) * pi.sign;", "s = (Vp > 0 ? 1 : -1);"),
    ("mu from the x component of the normal", "(i128)nmu * nmu * (nz * nz)",
     "(i128)nmu * nmu * (nx * nx)"),
    ("mu bin edge on the wrong side", "while (m > 0 && (i128)m * m * n2 > ",
     "while (m > 0 && (i128)m * m * n2 >= "),
    ("collinear triangles in the first mu bin", "int m = nmu;  // collinear", "int m = 0;  // collinear"),
    ("a cross-product term from the wrong side", "const i128 ny = (i128)u[2] * v[0] - (i128)u[0] * v[2];",
     "const i128 ny = (i128)u[2] * v[0] - (i128)u[0] * v[1];"),
]


def compile_variant(tmp, name, text):
    src = os.path.join(tmp, name + ".cpp")
    lib = os.path.join(tmp, name + ".so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", lib, src])
    return lib


def run_pins(lib):
    env = dict(os.environ, GS_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider", *PINS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = open(SRC).read()
    variants = {"unmodified": base}
    for k, (name, old, new) in enumerate(MUTANTS):
        assert base.count(old) == 1, name
        variants[f"m{k:02d}"] = base.replace(old, new)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 2) as ex:
        libs = dict(zip(variants, ex.map(lambda kv: compile_variant(str(tmp_path), *kv),
                                         variants.items())))
        results = dict(zip(libs, ex.map(run_pins, libs.values())))
    rc, out = results.pop("unmodified")
    assert rc == 0, "the pins fail on the unmodified oracle:\n" + out
    survivors = [MUTANTS[int(k[1:])][0] for k, (rc, _) in results.items() if rc == 0]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"
