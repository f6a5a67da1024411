"""The tiling rule of tpfa_apply_noalloc, checked on the CPU.

tpfa_apply_noalloc keeps one partial sum per sweep block in a fixed
workspace of 16384 entries, so it lengthens the z-runs of tpfa_apply's
tiling until the block count fits and refuses grids whose single-run
tiling still does not.  The rule lives in a plain C++ header
(csrc/sweep_plan.h); this test compiles a small driver against it with the
host compiler and checks deep, wide and ordinary grids, including ones far
too large to allocate on a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_03452_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "sweep_plan.h"
int main() {
  long long nx, ny, nz;
  int sms;
  while (std::scanf("%lld %lld %lld %d", &nx, &ny, &nz, &sms) == 4) {
    tpfa::Grid g{nx, ny, nz, nx * ny, nx * ny * nz};
    tpfa::Sweep a = tpfa::plan_sweep(g, 4, 4, 0, sms);
    tpfa::Sweep s;
    bool ok = tpfa::plan_noalloc(g, sms, &s);
    tpfa::Sweep r = tpfa::plan_sweep(g, 4, 4, s.zc, sms);
    std::printf("%d %d %lld %d %lld %lld %lld\n", ok ? 1 : 0, s.zc, (long long)s.nblocks, a.zc,
                (long long)a.nblocks, (long long)r.nblocks, (long long)(r.nwx * r.nwy));
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("plan")
    src, exe = d / "plan.cpp", d / "plan"
    src.write_text(DRIVER)
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)])

    def run(cases):
        inp = "".join(f"{nx} {ny} {nz} {sms}\n" for nx, ny, nz, sms in cases)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True)
        rows = [list(map(int, line.split())) for line in out.stdout.strip().splitlines()]
        return [dict(ok=r[0], zc=r[1], blocks=r[2], apply_zc=r[3], apply_blocks=r[4],
                     blocks_at_zc=r[5], cols=r[6]) for r in rows]
    return run


def test_ordinary_grids_keep_tpfa_apply_tiling(planner):
    cases = [(95, 33, 20, 152), (256, 192, 64, 152), (1024, 1024, 256, 152), (1, 1, 1, 152),
             (512, 256, 128, 148)]
    for c, r in zip(cases, planner(cases)):
        assert r["ok"] == 1, c
        assert (r["zc"], r["blocks"]) == (r["apply_zc"], r["apply_blocks"]), c
        assert r["blocks"] <= 16384


def test_deep_grids_lengthen_the_runs_until_the_workspace_fits(planner):
    # ceil(nx/30) * ceil(ny/4) = 60,000 columns: 128-plane runs need 240,000
    # blocks at nz = 2048; one run per column needs 15,000
    cases = [(30 * 300, 4 * 200, 2048, 152), (30 * 100, 4 * 100, 4096, 152),
             (30 * 512, 4 * 128, 300, 152), (1000, 1000, 100000, 152)]
    for c, r in zip(cases, planner(cases)):
        nx, ny, nz, _ = c
        assert r["apply_blocks"] > 16384, c       # tpfa_apply's own tiling would not fit
        assert r["ok"] == 1, c
        assert r["blocks"] <= 16384 and r["zc"] <= nz, (c, r)
        assert r["blocks"] == r["blocks_at_zc"], c  # exactly tpfa_apply's tiling at that run length
        assert r["zc"] == nz or r["zc"] in (256, 512, 1024, 2048, 4096, 8192, 16384, 32768,
                                              65536), (c, r)


def test_grids_that_cannot_fit_are_refused(planner):
    # more than 65,536 columns of warps: a single run per column is still too many blocks
    cases = [(30 * 1024, 4 * 128, 1, 152), (30 * 300, 4 * 300, 1024, 152), (30 * 512, 4 * 129, 7, 152)]
    for c, r in zip(cases, planner(cases)):
        assert r["cols"] > 65536, c
        assert r["ok"] == 0, c
        assert r["zc"] == c[2]  # it tried the whole column before refusing


def test_the_fit_limit_is_exact(planner):
    # exactly 65,536 columns in one run: 16,384 blocks of four warps
    r = planner([(30 * 512, 4 * 128, 1, 152), (30 * 512, 4 * 128, 1000, 152)])
    assert r[0]["ok"] == 1 and r[0]["blocks"] == 16384
    assert r[1]["ok"] == 1 and r[1]["zc"] == 1000 and r[1]["blocks"] == 16384
