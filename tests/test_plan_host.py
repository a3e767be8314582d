"""The block kernels' shared-memory plan (atm3_internal.cuh), host logic on
the CPU: a small program compiled against the header prints the plans of a
few launch shapes, and the pair rule's edge table must follow its capacity
parameter (1/16 edges per staged molecule): its size, the bytes it takes
(an edge-list word and a pair scalar per edge; 8-byte scalars in the
deterministic mode), the halving when it does not fit, and the FP32 rows
that carry the staged index (no index array).  No device is used."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_21230_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "atm3_internal.cuh"
using namespace atm3;
static void plan(const char* tag, int trav, int trunc, int prec, int mcap, int optin, int nw,
                 int det, int gpm16)
{
    AtmPlan P;
    const bool ok = atm_choose_plan_nw(trav, trunc, prec, mcap, optin, nw, P, det, gpm16);
    std::printf("%s %d %d %zu %d\n", tag, ok ? 1 : 0, P.gcap, P.smem, P.use_d);
}
int main()
{
    const int big = 232448;  // opt-in shared memory per block of the device
    for (int g : {256, 240, 200, 128})
        std::printf("g%d\n", g), plan("fp32", 2, 0, 1, 120, big, 4, 0, g);
    plan("fp32det", 2, 0, 1, 120, big, 4, 1, 256);
    plan("fp32det240", 2, 0, 1, 120, big, 4, 1, 240);
    plan("fp32small", 2, 0, 1, 120, 4096 + 15000, 4, 0, 256);
    plan("fp64", 2, 0, 0, 120, big, 8, 0, 256);
    plan("fp64g240", 2, 0, 0, 120, big, 8, 0, 240);
    plan("tiny", 2, 0, 1, 10, big, 4, 0, 256);
    const BlockSmem s32 = block_smem_plan<float>(0, 120, 4, 1920, 0, 0, 0);
    const BlockSmem s64 = block_smem_plan<double>(0, 120, 8, 1920, 0, 0, 0);
    std::printf("idx32 %zu\nidx64 %zu\n", s32.off_slot - s32.off_idx, s64.off_slot - s64.off_idx);
    return 0;
}
"""


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if nvcc is None:
        pytest.skip("no nvcc")
    d = tmp_path_factory.mktemp("plan")
    src = d / "plan.cu"
    src.write_text(PROGRAM)
    exe = d / "plan"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        p = line.split()
        if len(p) == 5:
            res[p[0] if p[0] != "fp32" else "fp32_%d" % res["_g"]] = dict(
                ok=int(p[1]), gcap=int(p[2]), smem=int(p[3]), use_d=int(p[4]))
        elif len(p) == 1:
            res["_g"] = int(p[0][1:])
        else:
            res[p[0]] = int(p[1])
    return res


def test_edge_table_follows_the_capacity_parameter(plans):
    m = 120
    for g in (256, 240, 200, 128):
        p = plans["fp32_%d" % g]
        assert p["ok"] == 1
        assert p["gcap"] == (g * m + 15) // 16
    # an edge-list word and an FP32 pair scalar per edge (segments padded to 16 bytes)
    d = plans["fp32_256"]["smem"] - plans["fp32_240"]["smem"]
    dg = plans["fp32_256"]["gcap"] - plans["fp32_240"]["gcap"]
    assert abs(d - 8 * dg) <= 32


def test_deterministic_scalars_take_eight_bytes(plans):
    dg = plans["fp32det"]["gcap"] - plans["fp32det240"]["gcap"]
    d = plans["fp32det"]["smem"] - plans["fp32det240"]["smem"]
    assert dg == 120 and abs(d - 12 * dg) <= 32   # 4-byte list word + 8-byte scalar


def test_table_halves_until_it_fits(plans):
    # (the pair scalars' segment also holds the per-molecule fallback
    # accumulators, 24 bytes per staged molecule, so it never shrinks below those)
    p = plans["fp32small"]
    assert p["ok"] == 1 and p["smem"] <= 15000
    assert p["gcap"] in (1920 // 2, 1920 // 4, 1920 // 8, 1920 // 16)
    assert plans["fp32_256"]["smem"] > 15000


def test_small_units_cap_the_table_at_their_pairs(plans):
    assert plans["tiny"]["gcap"] == 10 * 9 // 2


def test_fp64_table_and_index_array(plans):
    assert plans["fp64"]["ok"] == 1 and plans["fp64g240"]["ok"] == 1
    assert plans["fp64g240"]["gcap"] == (240 * 120 + 15) // 16
    assert plans["idx32"] == 0              # FP32: the index rides in the position rows
    assert plans["idx64"] >= 4 * 120        # FP64: an index array
