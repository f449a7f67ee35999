"""The bench's roofline counts come from FLOPS.md, and FLOPS.md's rows add up."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bench_reads_flops_md():
    b = _bench()
    f = b.read_flops()
    assert b.FLOPS_TT == f["FLOPS_TT"] == 106
    assert b.FLOPS_FUSED == f["FLOPS_FUSED"] == 147
    assert b.FLOPS_SYM == f["FLOPS_SYM"] == 135
    assert f["MUFU_PER_PAIR"] == 2


def test_flops_md_totals():
    f = _bench().read_flops()
    assert f["FLOPS_TT"] == f["FLOPS_GEOM"] + f["FLOPS_COEF_TT"] + f["FLOPS_APPLY_TT"]
    assert f["FLOPS_FUSED"] == f["FLOPS_TT"] + f["FLOPS_TR"]
    assert f["FLOPS_SYM"] == (f["FLOPS_GEOM"] + f["FLOPS_COEF_TT"] + f["FLOPS_SYM_FOLD"] + f["FLOPS_SYM_APPLY_T"] +
                              f["FLOPS_SYM_APPLY_S"])
    assert f["FLOPS_SYM_FUSED"] == f["FLOPS_SYM"] + f["FLOPS_SYM_TR"]
    assert f["FLOPS_SYM_RHS2"] == f["FLOPS_SYM_APPLY_T"] + f["FLOPS_SYM_APPLY_S"]
