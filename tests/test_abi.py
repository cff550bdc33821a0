"""The C-ABI library loads and exports every entry point declared in include/lbmpen.h
(no compute: runs without a GPU)."""
import ctypes
import os
import re

from paper_2511_01629_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbmpen.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lbm_create", "lbm_add_particles", "lbm_step", "lbm_get_fields",
              "lbm_get_particles", "lbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lbm.build()
    L = ctypes.CDLL(lbm.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_config_defaults_without_gpu():
    cfg = lbm.make_config(lbm.LBM_D2Q9, (100, 200, 1), bc=(lbm.LBM_PERIODIC, lbm.LBM_WALL), tau=0.8)
    assert cfg.n[0] == 100 and cfg.n[1] == 200 and cfg.n[2] == 1
    assert abs(cfg.alpha - 1.25) < 1e-15 and cfg.K == 1 and cfg.fp16_scale_log2 == 14
    assert lbm.lib().lbm_status_string(-4) == b"diverged"
