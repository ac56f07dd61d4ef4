"""The oracle under host AddressSanitizer and UndefinedBehaviorSanitizer.

A small C driver links `oracle/dbscan_oracle.c` (single-threaded build) with
-fsanitize=address,undefined and runs it over empty, tiny, duplicate-heavy,
off-grid and random inputs in every label mode; any sanitizer report makes the
driver exit non-zero.  It also checks a few results that need no reference:
min_pts = 1 makes every point core, min_pts > n makes every point noise.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(__file__)
ORACLE_C = os.path.join(HERE, "..", "oracle", "dbscan_oracle.c")

DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int oracle_dbscan(const float *x, int64_t n, int32_t d, float eps, int32_t min_pts, int32_t label_mode,
                  int32_t *labels, int32_t *counts_out, uint8_t *core_out, int32_t nthreads, int32_t mutation);

static uint64_t s = 88172645463325252ull;
static uint32_t rnd(void) { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return (uint32_t)s; }

static int run(int64_t n, int32_t d, float eps, int32_t min_pts, int mode, int dup, int offgrid) {
    float *x = malloc(sizeof(float) * (size_t)(n > 0 ? n : 1) * d);
    int32_t *lab = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *cnt = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *core = malloc((size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n * d; ++i) {
        uint32_t u = rnd() % (dup ? 8u : 1024u);
        x[i] = (float)u / 1024.0f;
    }
    if (offgrid && n > 0) x[0] = 0.3f;
    const int st = oracle_dbscan(x, n, d, eps, min_pts, mode, lab, cnt, core, 1, 0);
    int bad = 0;
    if (!offgrid && st == 0) {
        for (int64_t i = 0; i < n; ++i) {
            if (cnt[i] < 1) bad = 1;                     /* a point counts itself */
            if (min_pts == 1 && !core[i]) bad = 1;       /* every point is core */
            if (min_pts > n && lab[i] != -1) bad = 1;    /* every point is noise */
            if (lab[i] < -1 || lab[i] >= n) bad = 1;
        }
    }
    if (offgrid && st == 0) bad = 1;                     /* off-grid input is rejected */
    free(x); free(lab); free(cnt); free(core);
    return bad;
}

int main(void) {
    int bad = 0;
    for (int mode = 0; mode < 2; ++mode) {
        bad |= run(0, 2, 0.01f, 3, mode, 0, 0);
        bad |= run(1, 1, 0.01f, 1, mode, 0, 0);
        bad |= run(2, 3, 0.5f, 2, mode, 0, 0);
        bad |= run(300, 2, 0.02f, 4, mode, 0, 0);
        bad |= run(300, 2, 0.02f, 1, mode, 0, 0);
        bad |= run(300, 3, 0.02f, 400, mode, 0, 0);
        bad |= run(500, 2, 0.005f, 5, mode, 1, 0);     /* heavy duplicates */
        bad |= run(200, 64, 0.6f, 6, mode, 0, 0);
        bad |= run(50, 2, 0.02f, 3, mode, 0, 1);       /* off-grid */
    }
    if (bad) fprintf(stderr, "oracle property check failed\n");
    return bad;
}
"""


def test_oracle_clean_under_asan_and_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    drv = tmp_path / "driver.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "oracle_san"
    cc = ["gcc", "-std=c11", "-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer",
          "-fno-sanitize-recover=all", str(drv), ORACLE_C, "-o", str(exe), "-lm"]
    r = subprocess.run(cc, capture_output=True, text=True)
    if r.returncode != 0 and "asan" in (r.stderr or "").lower():
        pytest.skip("sanitizer runtime unavailable: " + r.stderr.strip().splitlines()[-1])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    out = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr[-3000:]
