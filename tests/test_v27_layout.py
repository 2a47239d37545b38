"""Host-side checks (no GPU) of the structured 27-point operator's layout
constants, compiled from the library's internal header with g++: the 13
forward offsets with their negatives and the centre cover {-1,0,1}^3 once,
the zero halo around the coefficient arrays and ring vectors covers the
largest offset plus a 16-byte-rounded copy, the tile header holds the
mbarriers (and, where the backward coefficients come through L2, the 13
backward-load pointers) with the slots 16-byte aligned after it, the
buffers are followed by one 40-byte copy plan per slot, and two CTAs' tiles
fit one SM's shared memory for every l, for the p(l)-CG and the classic CG
tiles in the layout each uses."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMEM_PER_SM = 228 * 1024          # GB300: shared memory per SM
SMEM_RESERVED_PER_CTA = 1024      # reserved by the runtime per resident CTA
STATIC_SMEM_BOUND = 8 * 1024      # the solver's static shared state stays below this


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("v27")
    src = d / "v27.cpp"
    src.write_text(r'''
#include <cstddef>
#include <cstdio>
#include "plcg_internal.h"
using namespace plcg;
int main() {
    for (int k = 0; k < 13; ++k) printf("dir %d %d %d\n", v27_dz(k), v27_dy(k), v27_dx(k));
    const long long g[][2] = {{1, 1}, {3, 5}, {128, 128}, {255, 3}, {1000, 7}, {5, 1000}};
    for (auto &p : g) printf("halo %lld %lld %lld\n", p[0], p[1], (long long)v27_halo(p[0], p[1]));
    for (int sb = 0; sb < 2; ++sb) {
        printf("layout %d %d %d %u\n", sb, v27_bufs(sb), v27_op_slots(sb), v27_hdr(sb));
        for (int l = 0; l <= 8; ++l)   // l = 0: classic CG's tiles (no vector slots)
            for (int j = 0; j < 2; ++j)
                printf("tile %d %d %d %d %u\n", sb, l, j, l ? v27_vec_slots(l, j) : 0,
                       v27_tile_bytes_nv(4, l ? v27_vec_slots(l, j) : 0, sb));
    }
    printf("slot %d\n", kV27Slot);
    printf("choice %d %d\n", (int)kV27StageBwdPlcg, (int)kV27StageBwdCg);
    printf("used %u %u %u %u\n", v27_tile_bytes(4, 1, true), v27_tile_bytes_nv(4, v27_vec_slots(1, true), kV27StageBwdPlcg),
           v27_tile_bytes_cg(4), v27_tile_bytes_nv(4, 0, kV27StageBwdCg));
    return 0;
}
''')
    exe = d / "v27"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.join(ROOT, "paper_1905_06850_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [line.split() for line in out.splitlines()]


def test_forward_offsets_cover_the_27_point_neighbourhood(values):
    fwd = [tuple(int(v) for v in r[1:]) for r in values if r[0] == "dir"]
    assert len(fwd) == 13 and len(set(fwd)) == 13
    nx, ny = 7, 5
    for dz, dy, dx in fwd:   # forward: a positive linear offset on any grid
        assert dz * nx * ny + dy * nx + dx > 0
    allo = set(fwd) | {(-a, -b, -c) for a, b, c in fwd} | {(0, 0, 0)}
    assert allo == {(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}


def test_halo_covers_the_largest_offset_and_rounding(values):
    for r in values:
        if r[0] != "halo":
            continue
        nx, ny, h = int(r[1]), int(r[2]), int(r[3])
        assert h % 64 == 0                     # whole 256-byte groups in FP32
        assert h >= nx * ny + nx + 1 + 4       # largest offset + a 16-byte rounding


def test_two_ctas_of_tiles_fit_one_sm(values):
    slot = next(int(r[1]) for r in values if r[0] == "slot")
    assert slot >= 256 + 2 + 3 and slot * 4 % 16 == 0   # a unit, z's x +- 1, the shift
    lay = {int(r[1]): (int(r[2]), int(r[3]), int(r[4])) for r in values if r[0] == "layout"}
    choice = [int(v) for v in next(r for r in values if r[0] == "choice")[1:]]
    for sb, (nbuf, ops, hdr) in lay.items():
        assert ops == 14 + 9 + (13 if sb else 0)   # diagonal + 13 forward, 9 z lines (+13 backward)
        assert hdr % 16 == 0 and hdr >= 16 * ((nbuf + 1) // 2) + (0 if sb else 13 * 8)
        assert nbuf >= 2
    for r in values:
        if r[0] != "tile":
            continue
        sb, l, jac, nv, tb = int(r[1]), int(r[2]), int(r[3]), int(r[4]), int(r[5])
        nbuf, ops, hdr = lay[sb]
        assert nv == (2 * l + 3 + jac if 1 <= l <= 3 else 0)
        assert tb == hdr + nbuf * (ops + nv) * slot * 4 + 40 * (ops + nv)   # + one copy plan per slot
        if sb == (choice[1] if l == 0 else choice[0]):   # the layouts the kernels use
            assert 2 * (tb + STATIC_SMEM_BOUND + SMEM_RESERVED_PER_CTA) <= SMEM_PER_SM, (sb, l, jac, tb)
    used = [int(v) for v in next(r for r in values if r[0] == "used")[1:]]
    assert used[0] == used[1] and used[2] == used[3]   # the kernels' sizes are the chosen layouts'
