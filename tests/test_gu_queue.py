"""Work queue of the FP32 phase's persistent g-and-update kernel (gu_item in
csrc/lgf_kernels.cuh), checked on the host: for every pair of supported extents
(Lz, Lt) and every lag 1..Lt, the 2 Lz Lt items are each build and each update of
every xy-plane exactly once, and every update of plane (z, t) comes after the
builds of (z, t), (z+1, t) and (z, t+1) (periodic) - the order that lets an
update wait for its builds without deadlock.  The function is compiled from the
library's own header by nvcc into a host program (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1301_3460_gb300", "csrc")

PROGRAM = r'''
#include <cstdio>
#include <vector>
#include "lgf_kernels.cuh"
int main()
{
    const int lens[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128};
    long checked = 0;
    for (int Lz : lens)
        for (int Lt : lens)
            for (int lag = 1; lag <= Lt; lag++) {
                const int np = Lz * Lt, n = 2 * np;
                std::vector<int> pos_build(np, -1), pos_update(np, -1);
                for (int i = 0; i < n; i++) {
                    const lgf::GuItem it = lgf::gu_item(i, Lz, Lt, lag);
                    if (it.plane < 0 || it.plane >= np) { printf("BAD plane %d %d %d %d\n", Lz, Lt, lag, i); return 1; }
                    std::vector<int>& pos = it.build ? pos_build : pos_update;
                    if (pos[it.plane] >= 0) { printf("BAD twice %d %d %d %d\n", Lz, Lt, lag, i); return 1; }
                    pos[it.plane] = i;
                }
                for (int p = 0; p < np; p++) {
                    if (pos_build[p] < 0 || pos_update[p] < 0) { printf("BAD missing %d %d %d\n", Lz, Lt, lag); return 1; }
                    const int z = p % Lz, t = p / Lz;
                    const int dep[3] = {p, (z + 1) % Lz + Lz * t, z + Lz * ((t + 1) % Lt)};
                    for (int d : dep)
                        if (!(pos_build[d] < pos_update[p])) { printf("BAD order %d %d %d %d\n", Lz, Lt, lag, p); return 1; }
                }
                checked++;
            }
    printf("OK %ld\n", checked);
    return 0;
}
'''


def test_queue_order_on_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "queue.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "queue"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                        "-I", CSRC, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
    lens = (4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128)
    assert int(out.stdout.split()[1]) == len(lens) * sum(lens)
