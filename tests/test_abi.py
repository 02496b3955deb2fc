"""The C interface: the library builds, loads without a GPU and exports every
entry point that include/pmgfr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pmgfr.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pmg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1908_03972_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("pmg_create", "pmg_upload_mesh", "pmg_set_state", "pmg_residual", "pmg_assemble_blocks",
                     "pmg_factor_blocks", "pmg_vcycle", "pmg_esdirk_step", "pmg_destroy", "pmg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1908_03972_gb300 import pmgfr
    missing = [n for n in declared_entry_points() if not hasattr(pmgfr, n)]
    assert not missing, missing


def test_binding_struct_layout_matches_header():
    from paper_1908_03972_gb300 import pmgfr
    # pmg_config: 1 int, 2 x int[8], 3 doubles, 1 int, 3 doubles, 4 ints, 3 doubles, 2 x double[4],
    # 1 int (+4 padding), 2 doubles, 3 ints (+4 padding), 1 double, 2 ints, 2 x double[5] (C layout)
    assert ctypes.sizeof(pmgfr.pmg_config) == (4 + 64 + 4 + 24 + 4 + 4 + 24 + 16 + 8 + 16 + 32 + 32 + 8 + 16 + 16 + 8 + 8
                                               + 80)
    assert pmgfr.pmg_config.copy_wait_s.offset == 272
    assert pmgfr.pmg_config.device_loop.offset == 280
    assert pmgfr.pmg_config.dim.offset == 284
    assert pmgfr.pmg_config.res_scale3.offset == 288
    assert ctypes.sizeof(pmgfr.pmg_mesh) == 24


def _cfg(**over):
    from paper_1908_03972_gb300 import pmgfr
    cfg = pmgfr.make_config([2, 1, 0], [1, 1, 1])
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("field,value", [("flux_prec", 3), ("block_prec", 3), ("esdirk_order", 5),
                                         ("n_levels", 0), ("gamma", 1.0), ("mu", -1.0), ("cfl_mode", 1)])
def test_create_rejects_invalid_configs_before_touching_the_gpu(lib, field, value):
    """pmg_create validates its configuration first: these fail with
    PMG_EINVAL on any machine (cfl_mode = 1 with cfl_init = 0)."""
    from paper_1908_03972_gb300 import pmgfr
    cfg = _cfg(**{field: value}, **({"cfl_init": 0.0} if field == "cfl_mode" else {}))
    with pytest.raises(pmgfr.PmgError) as ei:
        pmgfr.pmg_create(cfg)
    assert ei.value.status == pmgfr.PMG_EINVAL


def test_create_without_a_gpu_fails_instead_of_falling_back(lib):
    """No CPU fallback: a valid configuration without a CUDA device is
    PMG_ECUDA."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1908_03972_gb300 import pmgfr
    with pytest.raises(pmgfr.PmgError) as ei:
        pmgfr.pmg_create(_cfg())
    assert ei.value.status == pmgfr.PMG_ECUDA


def test_nk_structs_match_the_c_compiler(tmp_path):
    """pmg_nk_options / pmg_nk_stats: sizes and offsets from gcc on the header
    against the binding's ctypes structures."""
    import shutil
    import subprocess
    from paper_1908_03972_gb300 import pmgfr
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    fields = [f for f, _ in pmgfr.pmg_nk_options._fields_]
    prog = tmp_path / "lay.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{os.path.join(ROOT, "include", "pmgfr.h")}"',
             "int main(void) {", 'printf("%zu %zu\\n", sizeof(pmg_nk_options), sizeof(pmg_nk_stats));']
    lines += [f'printf("%zu\\n", offsetof(pmg_nk_options, {f}));' for f in fields]
    lines += ["return 0; }"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-std=c99", str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(pmgfr.pmg_nk_options)
    assert int(out[1]) == ctypes.sizeof(pmgfr.pmg_nk_stats)
    assert [int(x) for x in out[2:]] == [getattr(pmgfr.pmg_nk_options, f).offset for f in fields]
