"""The oracle's pins catch plausible mistakes: each case plants one mistake
in a copy of oracle.c (a dropped term, a wrong constant, index or operand),
rebuilds that copy and checks that the pin file covering it now fails.

Runs on the CPU only; the planted copies live in a temporary directory and
never touch the repository's oracle.
"""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text, planted text, pin file that must fail)
MUTANTS = [
    ("philox key schedule", "k1 += OR_PHILOX_W1;", "k1 += OR_PHILOX_W0;", "test_oracle_philox.py"),
    ("philox word order", "uint32_t n1 = lo1;", "uint32_t n1 = lo0;", "test_oracle_philox.py"),
    ("holes counted as bad", "if (d == -1) nholes++;", "if (d == -2) nholes++;", "test_oracle_partition.py"),
    ("zipf weight index", "partial += pow((double)(k + 1), -s);", "partial += pow((double)(k + 2), -s);",
     "test_oracle_c1.py"),
    ("update word", "w[13] ^= r[2];", "w[13] ^= r[1];", "test_oracle_c1.py"),
    ("hop counter", "w[15] += 1u;", "w[15] += 0u;", "test_oracle_c1.py"),
    ("destination word", "w[14] = (uint32_t)d;", "w[12] = (uint32_t)d;", "test_oracle_c1.py"),
    ("retire threshold", "#define OR_C1_RETIRE_THRESHOLD 429496730u",
     "#define OR_C1_RETIRE_THRESHOLD 529496730u", "test_oracle_c1.py"),
    ("voxel centre", "float u[3] = {px - 0.5f, py - 0.5f, pz - 0.5f};", "float u[3] = {px, py, pz};",
     "test_oracle_c0.py"),
    ("march step", "acc = acc + or_c0_sample(vol, N, px, py, pz) * 0.5f;",
     "acc = acc + or_c0_sample(vol, N, px, py, pz) * 0.25f;", "test_oracle_c0.py"),
    ("rk4 stage weight", "float s = ((k1[a] + 2.0f * k2[a]) + 2.0f * k3[a]) + k4[a];",
     "float s = ((k1[a] + 2.0f * k2[a]) + 1.0f * k3[a]) + k4[a];", "test_oracle_c2.py"),
    ("rk4 half step", "float half = h * 0.5f, sixth = h / 6.0f;", "float half = h * 0.25f, sixth = h / 6.0f;",
     "test_oracle_c2.py"),
    ("trilinear weight", "float c0 = c00 * gy + c10 * fr[1];", "float c0 = c00 * gx + c10 * fr[1];",
     "test_oracle_c2.py"),
    ("ea emission", "float cc = sg * 20.0f;", "float cc = sg * 10.0f;", "test_oracle_c3.py"),
    ("ea transmittance", "T = T * e;", "T = T * al;", "test_oracle_c3.py"),
    ("albedo", "if (!(or_u24(q4[2]) < 0.8f)) return 0;", "if (!(or_u24(q4[2]) < 0.6f)) return 0;",
     "test_oracle_c4.py"),
    ("hg asymmetry", "const float g = 0.3f;", "const float g = 0.5f;", "test_oracle_c4.py"),
    ("free flight", "float t = -logf(1.0f - or_u24(q4[0])) / sigmaMax;",
     "float t = -logf(1.0f - or_u24(q4[0])) / (2.0f * sigmaMax);", "test_oracle_c4.py"),
    ("migration axis", "b[0] = a[0] + a[3];", "b[0] = a[0] + a[4];", "test_oracle_mp.py"),
    ("tree weighted sum", "nd[1] += (uint64_t)a[6] * a[0];", "nd[1] += (uint64_t)a[6] * a[1];",
     "test_oracle_mp.py"),
    ("torus nearness", "if (d != 0 && d != 1 && d != g - 1) return 0;", "if (d != 0 && d != 1) return 0;",
     "test_oracle_mp.py"),
]


@pytest.fixture(scope="module")
def sandbox():
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    skip = shutil.ignore_patterns("*.so", "*.o", "__pycache__", "_build", "csrc")
    for sub in ("oracle", "tests", "paper_2605_30294_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=skip)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_the_originals_are_present():
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    for name, old, _, _ in MUTANTS:
        assert src.count(old) == 1, name


@pytest.mark.parametrize("name,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(sandbox, name, old, new, pin):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    path = os.path.join(sandbox, "oracle", "oracle.c")
    lib = os.path.join(sandbox, "oracle", "liboracle.so")
    try:
        open(path, "w").write(src.replace(old, new))
        if os.path.exists(lib):
            os.remove(lib)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join("tests", pin)], cwd=sandbox, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"{name}: {pin} still passes with the mistake planted"
    finally:
        open(path, "w").write(src)
        if os.path.exists(lib):
            os.remove(lib)
