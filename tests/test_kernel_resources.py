"""ptxas resources of the kernels a fwd+bwd step times (compiled here, no GPU):
the compositing kernels stay within the register budget their launch bounds
give (6 CTAs of 256 threads per SM for the forward, 4 of 256 for the
one-pixel backward, 7 of 128 for the two-pixel one), the backward does not
spill, and no timed kernel spills more than it does today.
A kernel edit that breaks one of these changes its speed before its results."""
import pytest

from paper_2312_02121_gb300 import build as gsbuild


def _have_nvcc() -> bool:
    try:
        gsbuild.nvcc()
        return True
    except RuntimeError:
        return False


pytestmark = pytest.mark.skipif(not _have_nvcc(), reason="needs the CUDA toolkit's nvcc")


@pytest.fixture(scope="module")
def rows():
    return gsbuild.resources()


def _one(rows, prefix):
    hits = [r for r in rows if r["name"].split("(")[0].replace("void ", "") == prefix]
    assert len(hits) == 1, (prefix, [r["name"] for r in hits])
    return hits[0]


def test_timed_kernels_keep_their_register_budget_and_spills(rows):
    # (kernel with template arguments, register cap from its launch bounds, spill bytes allowed)
    timed = [
        ("gs::k_raster_fwd<float, true, false, false, false, false>", 65536 // (256 * 6), 0),
        ("gs::k_raster_fwd<float, true, false, false, false, true>", 65536 // (256 * 6), 0),
        ("gs::k_raster_bwd<float, true, true, false, false, 1, 96>", 65536 // (256 * 4), 0),
        ("gs::k_raster_bwd<float, true, true, false, false, 2, 64>", 65536 // (128 * 7), 0),
        ("gs::k_project_fwd<float>", 255, 0),
        ("gs::k_project_bwd<float, false>", 65536 // (256 * 4), 0),
        ("gs::k_project_bwd<float, true>", 65536 // (256 * 4), 0),
        ("gs::k_emit<true>", 255, 0),
        ("gs::k_tile_order_rank", 255, 0),
        ("gs::k_finalize", 255, 0),
        ("gs::k_depth_keys", 255, 0),
        ("gs::k_radix_scatter<16>", 255, 0),
        ("gs::k_radix_scatter<8>", 255, 0),
        ("gs::k_radix_hist<16>", 255, 0),
        ("gs::k_l2_loss<float>", 255, 0),
    ]
    for name, cap, spill in timed:
        r = _one(rows, name)
        assert r["regs"] <= cap, (name, r["regs"], cap)
        assert r["spill_st"] <= spill and r["spill_ld"] <= spill, (name, r["spill_st"], r["spill_ld"])


def test_every_kernel_is_listed_with_its_registers(rows):
    assert len(rows) > 100
    assert all(r["regs"] > 0 for r in rows)
    assert {r["tu"] for r in rows} >= {"gs_project.cu", "gs_sort.cu", "gs_raster.cu", "gs_raster_bwd2.cu", "gs_raster_nc.cu",
                                     "gs_train.cu"}
