"""The FP32 table position (csrc/table_index.cuh: sample index and bilinear
fraction of a scaled radius in the pre-sampled w-planes, Sec. 5.1.1)
compiled for the host and checked against its definition: ir = floor(s)
(or s - 1 with fr = 1 at an exact integer), fr = s - ir, clamped to the last
interval beyond the table.  The range s < 1/4 is the one a visibility on a
grid point reaches with its central tap."""
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1903_06555_gb300", "csrc")


def host_table_index(s, last):
    code = r"""
#include <cstdio>
#define PHI_HD
#include "table_index.cuh"
int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb"); FILE* g = fopen(argv[2], "wb");
  const int last = atoi(argv[3]);
  float s;
  while (fread(&s, 4, 1, f) == 1) {
    int ir; float fr;
    phi::table_index(s, last, static_cast<float>(last), ir, fr);
    fwrite(&ir, 4, 1, g); fwrite(&fr, 4, 1, g);
  }
  fclose(f); fclose(g);
  return 0;
}
"""
    tmp = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"phi_tix_{os.getpid()}")
    with open(tmp + ".cpp", "w") as f:
        f.write(code.replace("#include <cstdio>", "#include <cstdio>\n#include <cstdlib>"))
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-I", CSRC, tmp + ".cpp", "-o", tmp],
                   check=True)
    np.asarray(s, np.float32).tofile(tmp + ".in")
    subprocess.run([tmp, tmp + ".in", tmp + ".out", str(last)], check=True)
    raw = np.fromfile(tmp + ".out", np.uint8).reshape(-1, 8)
    for ext in (".cpp", ".in", ".out", ""):
        os.remove(tmp + ext)
    ir = raw[:, :4].copy().view(np.int32).ravel()
    fr = raw[:, 4:].copy().view(np.float32).ravel()
    return ir, fr


def test_table_index_is_floor_and_fraction():
    last = 4313                      # 4315 samples, as at table_tol 1e-4 on a 4096^2 grid
    rng = np.random.default_rng(0)
    s = np.concatenate([
        np.array([0.0, 1e-38, 1e-20, 1e-7, 0.1, 0.2499999, 0.25, 0.2500001, 0.4999999, 0.5,
                  0.75, 0.9999999, 1.0, 1.0000001, 2.0, 3.0, 4312.9995, 4313.0], np.float32),
        rng.random(200_000).astype(np.float32) * np.float32(0.25),   # central taps on grid points
        rng.random(200_000).astype(np.float32) * np.float32(last),
        np.arange(0, last, dtype=np.float32),                        # exact integers
    ])
    ir, fr = host_table_index(s, last)
    inside = s < last
    # exact reconstruction, index in range, fraction in [0, 1]
    assert np.all(ir[inside].astype(np.float64) + fr[inside] == s[inside].astype(np.float64))
    assert np.all((ir[inside] >= 0) & (ir[inside] <= last - 1))
    assert np.all((fr[inside] >= 0) & (fr[inside] <= 1))
    # floor(s), except an exact integer may take the interval below with fr = 1
    fl = np.floor(s[inside].astype(np.float64)).astype(np.int64)
    alt = (fr[inside] == 1) & (ir[inside] == fl - 1)
    assert np.all((ir[inside] == fl) | alt)
    # below 1/4 in particular (the case a half-integer sum would break)
    small = s < 0.25
    assert np.all(ir[small] == 0) and np.all(fr[small] == s[small])


def test_table_index_clamps_beyond_the_table():
    last = 100
    s = np.array([100.0, 100.5, 101.0, 5000.0, np.inf, np.nan], np.float32)
    ir, fr = host_table_index(s, last)
    assert np.all(ir == last)
    assert np.allclose(fr[:4], s[:4] - last)
    assert np.isinf(fr[4]) and np.isnan(fr[5])
