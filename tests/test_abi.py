"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function declared in include/*.h; the ctypes structures match the header."""
import ctypes
import glob
import os
import re

from tests.conftest import ROOT


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"\b(bgt_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2503_13961_gb300 import _abi
    lib = _abi.load()
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_fields_follow_the_header():
    from paper_2503_13961_gb300 import _abi
    text = open(os.path.join(ROOT, "include", "bgt.h")).read()
    for struct, cls in (("bgt_config", _abi.Config), ("bgt_camera", _abi.Camera), ("bgt_scene", _abi.Scene),
                        ("bgt_grads", _abi.Grads), ("bgt_prims", _abi.Prims), ("bgt_tuning", _abi.Tuning)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                name = re.sub(r"\[.*?\]", "", part.strip().split()[-1]).lstrip("*")
                fields.append(name)
        assert fields == [f[0] for f in cls._fields_], struct


def test_default_config_without_gpu():
    from paper_2503_13961_gb300 import _abi
    lib = _abi.load()
    cfg = _abi.Config()
    assert lib.bgt_default_config(ctypes.byref(cfg)) == 0
    assert cfg.degree == 2 and cfg.tess_level == 8 and cfg.tile_size == 16
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and abs(cfg.alpha_max - 0.99) < 1e-7
    assert lib.bgt_default_config(None) == 1
    # bad configurations are rejected on the host, before any CUDA call
    cfg.tile_size = 12
    h = ctypes.c_void_p()
    assert lib.bgt_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert not h.value


def test_product_path_has_no_oracle_dependency():
    # the package never imports, links or loads the oracle
    pkg = os.path.join(ROOT, "paper_2503_13961_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            assert not re.search(r"(from|import)\s+oracle|bgt_oracle|bgto_", src), f


def test_binding_rejects_host_tensors_before_any_call():
    # the library reads and writes these through device pointers: a host
    # tensor (or a wrong dtype, layout or size) is refused in Python first
    import pytest
    import torch
    from paper_2503_13961_gb300 import render as R
    for t in (torch.zeros(6), torch.zeros(6, dtype=torch.float64), torch.zeros(3, 2).t()):
        with pytest.raises(ValueError):
            R._device_f32(t, "x")
    assert R._device_f32(None, "x") is None


def test_prebuilt_camera_batch_equals_the_per_call_array():
    import ctypes
    from paper_2503_13961_gb300 import _abi, scenes
    from paper_2503_13961_gb300 import render as R
    _, cams = scenes.config_scene(4)
    batch = R.Cameras(cams)
    arr = _abi.camera_array(cams)
    assert len(batch) == len(cams) and R.view_pixels(batch) == R.view_pixels(list(cams))
    assert ctypes.string_at(batch.array, ctypes.sizeof(batch.array)) == ctypes.string_at(arr, ctypes.sizeof(arr))
