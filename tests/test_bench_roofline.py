"""The roofline object of bench.py's stencil line (host logic, no GPU): the
HBM fraction counts the algorithmic vector passes of the iteration in the
vector type plus two FP64 residual sweeps; the FP64 fraction counts the
flops the solve's kernel issues on the FP64 pipe -- 16 per row for the
headline kernel (FP64 p(1)-CG, scaled bases, two rows per thread, the
neighbour sum on the integer units), with the paper's 24 beside them -- and
the paper's count for the other FP64 kernels, and does not apply to FP32
sweeps; "bound" names the larger fraction; traffic scales the committed ncu
record's bytes per row and sweep."""
import pytest

import bench

N256 = 256 ** 3


def roof(**kw):
    args = dict(n=N256, nx=256, l=1, prec="fp64", iters=533, seconds=0.162, hbm_peak=6792.7,
                hbm_src="measured", dp_peak_tf=1.2552, dp_src="measured", rec=None)
    args.update(kw)
    return bench.stencil_roofline(**args)


def test_headline_counts_fp64_pipe_flops():
    r = roof()
    alu = r if r["bound"] == "alu" else r["alu"]
    hbm = r["hbm"] if r["bound"] == "alu" else r
    flops_pipe = 533 * 16 * N256 / 0.162 / 1e12
    assert alu["flops_per_row_iter"] == 16 and alu["paper_flops_per_row_iter"] == 24
    assert alu["achieved"] == pytest.approx(flops_pipe, rel=1e-3)
    assert alu["frac"] == pytest.approx(flops_pipe / 1.2552, rel=1e-3)
    assert alu["paper_flops_tflops"] == pytest.approx(flops_pipe * 24 / 16, rel=1e-3)
    byt = 533 * 10 * 8 * N256 + 3 * 8 * N256 * 2
    assert hbm["achieved"] == pytest.approx(byt / 0.162 / 1e9, rel=1e-3)
    assert hbm["frac"] == pytest.approx(byt / 0.162 / 1e9 / 6792.7, rel=1e-3)
    assert r["bound"] == ("alu" if alu["frac"] >= hbm["frac"] else "hbm")
    assert alu["frac"] < 1.0 and hbm["frac"] < 1.0


def test_other_kernels_keep_the_paper_count():
    for kw in ({"nx": 255, "n": 255 ** 3}, {"n": 64 ** 3, "nx": 64}, {"l": 2}):
        r = roof(**kw)
        alu = r if r["bound"] == "alu" else r["alu"]
        assert alu["flops_per_row_iter"] == 18 + 6 * kw.get("l", 1) and "flops_counted" not in alu


def test_fp32_counts_four_byte_vectors_against_hbm_only():
    r = roof(prec="fp32", seconds=0.062, iters=538)
    assert r["bound"] == "hbm" and "alu" not in r
    byt = 538 * 10 * 4 * N256 + 3 * 8 * N256 * 2
    assert r["achieved"] == pytest.approx(byt / 0.062 / 1e9, rel=1e-3)


def test_traffic_from_the_ncu_record():
    r = roof(rec={"dram_bytes_per_point_iter": 76.76, "fp64_pipe_pct": 64.8})
    assert r["traffic"] == round(76.76 * N256 * 535)
    alu = r if r["bound"] == "alu" else r["alu"]
    assert alu["ncu_fp64_pipe_pct"] == 64.8
    assert roof()["traffic"] is None
