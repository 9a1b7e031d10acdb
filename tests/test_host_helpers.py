"""Host-side helpers of the CUDA path, compiled for the CPU (no GPU).

The one-byte path code of |P_v| (internal.cuh) decides which candidates a hub
query may skip. Its exactness argument needs three properties, checked here
exhaustively up to 2^25 and at the top of the range:
  * path_code is monotone in the path count;
  * path_code(x) >= c exactly when x >= code_floor(c);
  * code_floor is strictly increasing, exact (code_floor(c) = c) below 128.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1504_02577_gb300", "csrc", "internal.cuh")

_HARNESS = r"""
#include "INTERNAL"
#include <cstdio>
int main() {
    for (uint32_t c = 0; c < 256; ++c) {
        if (c < 128 && code_floor(c) != (int64_t)c) { printf("floor(%u) != %u\n", c, c); return 1; }
        if (c > 0 && code_floor(c) <= code_floor(c - 1)) { printf("floor not increasing at %u\n", c); return 1; }
        if (path_code(code_floor(c)) != c) { printf("code(floor(%u)) != %u\n", c, c); return 1; }
    }
    uint32_t prev = 0;
    // every count below 2^25 (the top code starts at 15 * 2^19), then a few far above
    const int64_t top[] = {(int64_t)1 << 25, ((int64_t)1 << 26) + 3, (int64_t)1 << 40, INT64_MAX};
    for (int64_t i = 0; i < ((int64_t)1 << 25) + 4; ++i) {
        const int64_t x = i < ((int64_t)1 << 25) ? i : top[i - ((int64_t)1 << 25)];
        const uint32_t cx = path_code(x);
        if (cx > 255 || cx < prev) { printf("code not monotone at %lld\n", (long long)x); return 1; }
        prev = cx;
        if (code_floor(cx) > x) { printf("floor above x at %lld\n", (long long)x); return 1; }
        if (cx < 255 && code_floor(cx + 1) <= x) { printf("next floor not above x at %lld\n", (long long)x); return 1; }
    }
    if (path_code(-5) != 0) { printf("negative count\n"); return 1; }
    printf("ok\n");
    return 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_path_code_properties(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "code_check.cpp"
    src.write_text(_HARNESS.replace("INTERNAL", HEADER))
    exe = tmp_path / "code_check"
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{inc}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
