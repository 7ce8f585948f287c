"""Host logic of the GB300 validation module (no GPU): the estimator's description of the
validation kernels, the parsing of ncu's CSV logs and the volumes per lattice update that
the comparison reports."""
import json

import numpy as np

from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import validation as V
from paper_2204_14242_gb300 import workloads as W


def test_model_config_describes_the_kernels():
    v = {"kind": "star", "N": (64, 32, 16), "B": (32, 4, 1), "fold_axis": 0, "fold": 1, "r": 4}
    c = V.model_config(v, regs=40)
    src, dst = c.fields
    assert len(src.accesses) == 25 and all(not a.is_store for a in src.accesses)
    assert [a.is_store for a in dst.accesses] == [1]
    # element (x, y, z) of the padded array lies at (z + PAD) Sy Sx + (y + PAD) Sx + (x + PAD)
    sx, sy = 64 + 2 * V.PAD, (64 + 2 * V.PAD) * (32 + 2 * V.PAD)
    assert src.strides == (1, sx, sy) and src.const_off == V.PAD * (1 + sx + sy)
    assert c.flops_per_lup == 6 * 4 + 3 and c.regs_per_thread == 40
    lbm = V.model_config({"kind": "lbm", "N": (16, 16, 8), "B": (16, 4, 1), "fold_axis": 0, "fold": 1})
    assert len(lbm.fields) == 2 * 19
    # the host compiler accepts both (no device needed)
    info = B.ws_describe([c, lbm], W.gb300())
    assert (info["status"] == 0).all()


def test_ncu_csv_parsing_and_volumes(tmp_path):
    csv_path = tmp_path / "ncu.csv"
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"',
            '"0","star_kernel","dram__bytes_read.sum","Mbyte","2.5"',
            '"0","star_kernel","dram__bytes_write.sum","byte","1000000"',
            '"0","star_kernel","lts__t_sectors_srcunit_tex_op_read.sum","sector","250000"',
            '"0","star_kernel","gpu__time_duration.sum","usecond","50"']
    csv_path.write_text("==PROF== something\n" + "\n".join(rows) + "\n")
    m = V._ncu_rows([str(csv_path)])
    assert len(m) == 1
    assert m[0]["dram__bytes_read.sum"] == 2.5e6 and m[0]["dram__bytes_write.sum"] == 1e6
    assert np.isclose(m[0]["gpu__time_duration.sum"], 50e-6)
    pred = {"i": 0, "kind": "star", "B": [32, 4, 1], "fold_axis": 0, "fold": 1, "lups": 125000, "glups": 0,
            "pred": {"v_l2_load": 64.0, "v_dram_load": 20.0, "v_dram_store": 8.0, "glups": 2.0, "limiter": 2,
                     "t_pred": 1.0, "v_l1": 100.0, "blk_load_sectors": 10, "lups_block": 10, "o_l1": 0.5}}
    pred_path = tmp_path / "pred.json"
    pred_path.write_text(json.dumps(pred) + "\n")
    out = V.report(str(pred_path), [str(csv_path)])
    # 32 B x 250,000 sectors / 125,000 LUP = 64 B/LUP; 2.5 MB / 125,000 = 20; 1 MB / 125,000 = 8
    assert "| 64.0 / 64.0 |" in out and "| 20.0 / 20.0 |" in out and "| 8.0 / 8.0 |" in out
    assert "Median relative error: L2<-L1 load 0.00, DRAM load 0.00, DRAM store 0.00." in out


def test_rhat_limits():
    # R(O) = a exp(-b exp(-c O)) with c < 0: near a for small O, near 0 for large O
    p = (1.0, 0.01, -3.07)
    assert V._rhat(p, 0.0) > 0.98 and V._rhat(p, 5.0) < 1e-3
