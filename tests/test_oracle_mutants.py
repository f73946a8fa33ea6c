"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of
oracle/dm_oracle.c (a dropped term, an off-by-one, a wrong comparison, swapped axes),
builds it with gcc, and runs the CPU pin tests against that build; they must fail.  An
unaltered copy must pass.  Nothing here touches the GPU or the product library."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dm_oracle.c")
PINS = [os.path.join(ROOT, "tests", f) for f in
        ("test_oracle_pins.py", "test_oracle_properties.py", "test_rho_min_partition.py")]

# (name, text in the oracle, planted replacement)
MUTANTS = [
    ("DT keeps only the 6 face neighbours (dropped diagonal terms)",
     "if (!before) continue;",
     "if (!before || (dx != 0) + (dy != 0) + (dz != 0) > 1) continue;"),
    ("DT saturates at 254",
     "out[i] = (uint8_t)(d[i] > 255 ? 255 : d[i]);",
     "out[i] = (uint8_t)(d[i] > 254 ? 254 : d[i]);"),
    ("footprint loses one apron voxel on the low side",
     "*lo = c * b - a;",
     "*lo = c * b - a + 1;"),
    ("zero alpha counts as visible",
     "if (alpha > 0.0f) smask",
     "if (alpha >= 0.0f) smask"),
    ("uniform borders rounded up instead of down",
     "return ((int64_t)p * N) / K;",
     "return ((int64_t)p * N + K - 1) / K;"),
    ("combine skips the last partition",
     "for (int32_t p = 0; p < K; ++p) {\n        if (!((smask[p / 64] >> (p % 64)) & 1u)) continue;",
     "for (int32_t p = 0; p < K - 1; ++p) {\n        if (!((smask[p / 64] >> (p % 64)) & 1u)) continue;"),
    ("POM reads the volume with x and y swapped",
     "int64_t i = voxel_at(vol, bytes_per_voxel, (z * Y + y) * X + x, N);\n"
     "                            int32_t p = lut[i];",
     "int64_t i = voxel_at(vol, bytes_per_voxel, (z * X + x) * Y + y, N);\n"
     "                            int32_t p = lut[i];"),
    ("min/max occupancy leaves out the block maximum",
     "for (int64_t v = vmin[i]; v <= vmax[i] && v < N; ++v)",
     "for (int64_t v = vmin[i]; v < vmax[i] && v < N; ++v)"),
    ("intensities above the TF domain dropped instead of clamped",
     "return v > N - 1 ? N - 1 : v;",
     "return v > N - 1 ? 0 : v;"),
    ("shell search misses one face of each shell",
     "int on_shell = (dz == -r || dz == r || dy == -r || dy == r);",
     "int on_shell = (dz == -r || dz == r || dy == -r);"),
    ("grid rounds the block count down",
     "static int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }",
     "static int64_t cdiv(int64_t a, int64_t b) { return a / b > 0 ? a / b : 1; }"),
    ("POM sets every partition bit in the first mask word",
     "mask[blk * W + p / 64] |= (uint64_t)1 << (p % 64);",
     "mask[blk * W] |= (uint64_t)1 << (p % 64);"),
    ("exact occupancy counts zero alpha as visible",
     "if (tf_rgba[4 * i + 3] > 0.0f) o = 1;",
     "if (tf_rgba[4 * i + 3] >= 0.0f) o = 1;"),
    ("DT without its backward pass",
     "int after = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));",
     "int after = 0;"),
    ("footprint loses one apron voxel on the high side",
     "*hi = c * b + b - 1 + a;",
     "*hi = c * b + b - 2 + a;"),
    ("forward DT pass wraps from the end of a row to the start of the next",
     "if (nz < 0 || ny < 0 || ny >= gy || nx < 0 || nx >= gx) continue;",
     "if (nz < 0 || ny < 0 || ny >= gy || nx < 0) continue;"),
    ("shell search reports one more than the radius",
     "if (occ[(nz * gy + ny) * gx + nx]) return (int)r;",
     "if (occ[(nz * gy + ny) * gx + nx]) return (int)r + 1;"),
    ("shell search gives up one radius early",
     "for (int64_t r = 0; r < 255; ++r) {",
     "for (int64_t r = 0; r < 254; ++r) {"),
    ("an empty S combines to 0 instead of 255",
     "for (int64_t i = 0; i < G; ++i) out[i] = 255;",
     "for (int64_t i = 0; i < G; ++i) out[i] = 0;"),
]


def _run_pins(tmp_path, source):
    src = tmp_path / "dm_oracle.c"
    lib = tmp_path / "libdm_oracle.so"
    src.write_text(source)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(lib),
                           str(src)])
    env = dict(os.environ, DM_ORACLE_LIB=str(lib))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu",
                           "-p", "no:cacheprovider", *PINS], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_unaltered_copy_passes_the_pins(tmp_path):
    r = _run_pins(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_fail_on_a_planted_mistake(tmp_path, name, old, new):
    source = open(SRC).read()
    assert source.count(old) == 1, f"planting site not found once: {name}"
    r = _run_pins(tmp_path, source.replace(old, new))
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.stdout[-1500:])
