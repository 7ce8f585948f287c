"""The C-ABI library builds, loads and exports every entry point include/*.h declares
(CPU only: no compute call needs a GPU here)."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2204_14242_gb300 import _build
from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(ws_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    lib = _build.build()
    assert os.path.exists(lib)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    declared = declared_functions()
    assert len(declared) >= 20
    missing = declared - exported
    assert not missing, missing
    assert set(B.EXPORTS) <= exported
    B.load()  # loads and binds every signature


def test_struct_layouts_match_the_header():
    text = open(os.path.join(ROOT, "include", "warpspeed.h")).read()
    sizes = dict(re.findall(r"\}\s*(ws_\w+);\s*/\*\s*(\d+) bytes", text))
    assert int(sizes["ws_access"]) == B.ACCESS.itemsize
    assert int(sizes["ws_field"]) == B.FIELD.itemsize
    assert int(sizes["ws_config"]) == B.CONFIG.itemsize
    assert int(sizes["ws_hw"]) == B.HW.itemsize
    assert int(sizes["ws_result"]) == B.RESULT.itemsize
    assert int(sizes["ws_cfg_info"]) == B.CFG_INFO.itemsize
    assert int(sizes["ws_tuning"]) == B.TUNING.itemsize
    assert int(sizes["ws_profile"]) == B.PROFILE.itemsize
    assert int(sizes["ws_plan_summary"]) == B.PLAN_SUMMARY.itemsize
    assert int(sizes["ws_server_stats"]) == B.SERVER_STATS.itemsize
    assert int(sizes["ws_peaks"]) == 4 * 8


def test_host_constants_and_rank_key():
    assert B.ws_version() == 1
    lib = B.load()
    assert lib.ws_status_string(B.WS_ENOMEM).decode().startswith("does not fit")
    h = B.ws_hw_a100()[0]
    ref = B.hw_struct(W.a100())[0]
    for k in B.HW.names:
        assert np.array_equal(h[k], ref[k]), k
    rng = W.SplitMix64(9)
    for _ in range(2000):
        t = rng.uniform() * 10.0 ** rng.randint(-14, -8)
        assert B.ws_rank_key(t) == oracle.rank_key(t)
    for t in (0.0, float("inf"), 1.0 + 2.0 ** -41, 1.0 + 3 * 2.0 ** -41):
        assert B.ws_rank_key(t) == oracle.rank_key(t)


def test_context_creation_fails_cleanly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(B.WsError) as e:
        B.Context(0, 1 << 24, use_torch=False)
    assert e.value.code in (B.WS_ECUDA, B.WS_EINVAL)
