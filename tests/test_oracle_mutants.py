"""The oracle's pins have teeth: each plausible mistake planted in a copy of the
oracle source (on the CPU, in a temporary directory) must make the pin suite fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "px_oracle.cpp")

# (name, text in the oracle source, planted replacement)
MUTANTS = [
    ("hash_shift", "x ^= x >> 33;\n    x *= 0xff51afd7ed558ccdULL;", "x ^= x >> 31;\n    x *= 0xff51afd7ed558ccdULL;"),
    ("hash_constant", "0xc4ceb9fe1a85ec53ULL", "0xc4ceb9fe1a85ec55ULL"),
    ("part_low_bits", "((h >> 32) * static_cast<uint64_t>(nparts)) >> 32",
     "((h & 0xffffffffULL) * static_cast<uint64_t>(nparts)) >> 32"),
    ("part_no_seed", "orc_fmix64(static_cast<uint64_t>(key) ^ seed)", "orc_fmix64(static_cast<uint64_t>(key))"),
    ("filter_closed_hi", "lo <= v && v < hi", "lo <= v && v <= hi"),
    ("int8_unsigned", "static_cast<const int8_t*>(col)[i]", "static_cast<const uint8_t*>(col)[i]"),
    ("partition_unstable", "std::stable_sort(order.begin()", "std::sort(order.begin()"),
    ("partition_offsets_shift", "offsets[part[j] + 1] += 1;", "offsets[part[j]] += 1;"),
    ("join_first_match_only", "for (auto it = lo; it != sorted.end() && it->first == key; ++it) {",
     "for (auto it = lo; it != sorted.end() && it->first == key && it == lo; ++it) {"),
    ("join_segment_bounds", "const int64_t b1 = nsegs > 0 ? build_seg[q + 1] : nbuild;",
     "const int64_t b1 = nsegs > 0 ? build_seg[q + 1] - (q > 0) : nbuild;"),
    ("groupby_mul_to_add", "acc[a] += x * y;", "acc[a] += x + y;"),
    ("groupby_count_twice", "acc[a] += 1;", "acc[a] += 1 + (r == 3);"),
    ("groupby_segment_advance", "while (q + 1 < nsegs && j >= seg[q + 1]) ++q;",
     "while (q + 1 < nsegs && j > seg[q + 1]) ++q;"),
]


def test_every_planted_mistake_fails_the_pins(tmp_path):
    src = open(SRC).read()
    procs = []
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, f"mutant {name}: anchor text not found exactly once"
        mdir = tmp_path / name
        mdir.mkdir()
        cpp = mdir / "m.cpp"
        cpp.write_text(src.replace(old, new))
        lib = mdir / "libm.so"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(lib), str(cpp)])
        env = dict(os.environ, PX_ORACLE_LIB=str(lib))
        procs.append((name, subprocess.Popen(
            [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
             os.path.join(ROOT, "tests", "test_oracle_pins.py")],
            cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    survivors = []
    for name, p in procs:
        p.communicate(timeout=600)
        if p.returncode == 0:
            survivors.append(name)
    assert not survivors, f"pins did not catch planted mistakes: {survivors}"


# Mistakes planted in the oracle's Python compositions (oracle/__init__.py): the
# mutated package is copied to a temporary directory that shadows the real one.
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")
PY_MUTANTS = [
    ("fragment_price_from_build_row",
     '(SUM, d["price"][pr], None), (SUM_MUL, d["price"][pr], d["qty"][pr]),\n                         (COUNT',
     '(SUM, d["price"][br], None), (SUM_MUL, d["price"][pr], d["qty"][pr]),\n                         (COUNT'),
    ("fragment_filter_dropped", 'sel = filter(d["date"], lo, hi)\n    pr, br, _ = join(d["pk"], d["key"], sel=sel)',
     'sel = filter(d["date"], lo, hi)\n    pr, br, _ = join(d["pk"], d["key"], sel=None)'),
    ("wide_join_amount_from_build_row", '[(SUM, d["amount"][pr], None), (SUM_MUL, d["price"][pr], d["qty"][pr]),\n                            (COUNT',
     '[(SUM, d["amount"][br], None), (SUM_MUL, d["price"][pr], d["qty"][pr]),\n                            (COUNT'),
    ("final_counts_partials", '(SUM, partial["aggs"][1], None)])', '(COUNT, None, None)])'),
]


def test_every_planted_composition_mistake_fails_the_pins(tmp_path):
    import shutil
    src = open(PY_SRC).read()
    lib = tmp_path / "liboracle.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(lib), SRC])
    procs = []
    for name, old, new in PY_MUTANTS:
        assert src.count(old) == 1, f"mutant {name}: anchor text not found exactly once"
        pkg = tmp_path / name / "oracle"
        pkg.mkdir(parents=True)
        (pkg / "__init__.py").write_text(src.replace(old, new))
        tests = tmp_path / name / "tests"
        tests.mkdir()
        shutil.copy(os.path.join(ROOT, "tests", "test_oracle_pins.py"), tests / "test_oracle_pins.py")
        env = dict(os.environ, PX_ORACLE_LIB=str(lib),
                   PYTHONPATH=os.pathsep.join([str(tmp_path / name), ROOT]))
        procs.append((name, subprocess.Popen(
            [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--rootdir", str(tmp_path / name),
             str(tests / "test_oracle_pins.py")],
            cwd=str(tmp_path / name), env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    survivors = []
    for name, p in procs:
        out, _ = p.communicate(timeout=600)
        if p.returncode == 0:
            survivors.append(name)
        elif b"ModuleNotFoundError" in out or b"ImportError" in out:
            survivors.append(name + " (did not import)")
    assert not survivors, f"pins did not catch planted mistakes: {survivors}"


def test_copied_oracle_package_passes_the_pins_unmutated(tmp_path):
    # The harness above is sound: the same copy without a mutation passes.
    import shutil
    lib = tmp_path / "liboracle.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(lib), SRC])
    pkg = tmp_path / "clean" / "oracle"
    pkg.mkdir(parents=True)
    shutil.copy(PY_SRC, pkg / "__init__.py")
    tests = tmp_path / "clean" / "tests"
    tests.mkdir()
    shutil.copy(os.path.join(ROOT, "tests", "test_oracle_pins.py"), tests / "test_oracle_pins.py")
    env = dict(os.environ, PX_ORACLE_LIB=str(lib), PYTHONPATH=os.pathsep.join([str(tmp_path / "clean"), ROOT]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--rootdir",
                        str(tmp_path / "clean"), str(tests / "test_oracle_pins.py")],
                       cwd=str(tmp_path / "clean"), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
    import_check = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"],
                                  cwd=str(tmp_path / "clean"), env=env, capture_output=True, text=True)
    assert str(tmp_path / "clean") in import_check.stdout
