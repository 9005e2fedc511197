"""The C ABI libraries build for sm_103a, load, and export every entry point
that include/lbm_ewod.h and include/unet_bf16.h declare (no GPU needed:
nothing is called that touches a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_ewod.h")
UNET_HEADER = os.path.join(ROOT, "include", "unet_bf16.h")


def declared_functions(header=HEADER, prefix="lbm_"):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0708_4182_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(f"nvcc unavailable: {e}")
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_workspace_bytes", "lbm_create", "lbm_set_geometry", "lbm_set_field",
                     "lbm_get_field", "lbm_step", "lbm_observables", "lbm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_every_unet_symbol_is_exported(lib):
    from paper_0708_4182_gb300 import build
    unet = ctypes.CDLL(build.UNET_LIB)
    names = declared_functions(UNET_HEADER, "unet_")
    assert "unet_conv3x3" in names and "unet_conv_pack" in names and "unet_adam" in names
    for name in names:
        assert hasattr(unet, name), name


def test_host_only_entry_points(lib):
    """Entry points that touch no device: workspace sizing, status strings."""
    from paper_0708_4182_gb300 import lbm
    p = lbm.make_params(128, 64)
    assert lbm.lbm_workspace_bytes(p) > 2 * 9 * 64 * 128 * 4
    assert lbm.lbm_workspace_bytes(lbm.make_params(128, 64, tau=0.4)) == 0
    assert lbm.lbm_workspace_bytes(lbm.make_params(128, 64, tile_rows=3)) == 0
    assert lbm.lbm_workspace_bytes(lbm.make_params(128, 64, storage=9)) == 0
    assert lbm.lbm_workspace_bytes(lbm.make_params(128, 300000)) == 0
    assert lbm.lbm_status_string(lbm.LBM_ESTATE) == "LBM_ESTATE"
    assert lbm.lbm_last_error(None) == "null context"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_0708_4182_gb300 import build, lbm
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lbm, "_lib", None)
    with pytest.raises(lbm.LbmUnavailable):
        lbm.load()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_0708_4182_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "lbm_oracle" not in text, fn
