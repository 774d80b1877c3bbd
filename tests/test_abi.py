"""CPU checks of the C ABI: the library builds, loads without a GPU, exports every
function include/agents.h declares, its structs have the header's layout, defaults are the
paper's constants, and parameter validation rejects bad input before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2510_16154_gb300 import lib
from paper_2510_16154_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "agents.h")
HEADERS = [HEADER, os.path.join(ROOT, "include", "warmstart.h")]


@pytest.fixture(scope="module")
def cdll():
    build()
    return lib.load()


def _declared_functions(headers=(HEADER,)):
    text = "".join(open(h).read() for h in headers)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_six_entry_points():
    names = _declared_functions()
    for required in ["agents_init", "agents_forward", "agents_adjoint", "pd_tv_step",
                     "alm_update", "solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(cdll):
    names = _declared_functions(HEADERS)
    assert len(names) >= 12
    for name in names:
        assert hasattr(cdll, name), name
        assert name in lib._SIGNATURES, f"binding lacks {name}"


def test_struct_layouts_match_header():
    # int32 x5, pad, double x4, double[2] x2, int32 x3, pad -> 88 bytes
    assert ctypes.sizeof(lib.agents_params) == 5 * 4 + 4 + 8 * 4 + 16 * 2 + 3 * 4 + 4
    assert lib.agents_params.dt.offset == 24
    assert ctypes.sizeof(lib.agents_solve_opts) == 3 * 4 + 4 + 4 * 8
    assert ctypes.sizeof(lib.agents_solve_info) == 5 * 4 + 4 + 3 * 8 + 4 * 8 + 8
    assert ctypes.sizeof(lib.agents_iter_record) == 4 * 4 + 4 * 8
    assert ctypes.sizeof(lib.agents_outer_record) == 2 * 4 + 8 * 8


def test_paper_defaults(cdll):
    p = lib.agents_default_params(64, 48, 3, 2, 20)
    assert (p.height, p.width, p.channels, p.radius, p.nsteps) == (64, 48, 3, 2, 20)
    assert p.dt == 0.25 and p.rho == 1e-2 and p.gamma == 1e-2 and p.alpha == 3000.0
    assert tuple(p.eps_lo) == (2.0, 2.0) and tuple(p.eps_hi) == (1100.0, 1100.0)
    o = lib.agents_default_solve_opts()
    assert o.sigma0 == 1.0 and o.ls_b == 0.5 and o.ls_c == 1e-4 and o.max_ls == 30


@pytest.mark.parametrize("field,value", [("height", 0), ("channels", 0), ("channels", 65),
                                         ("radius", 0), ("nsteps", 0), ("dt", 0.0),
                                         ("rho", -1.0), ("norm_mode", 2), ("tv_mode", 5),
                                         ("traj_mode", -1)])
def test_validation_rejects_bad_params(cdll, field, value):
    p = lib.agents_default_params(8, 8, 3, 2, 4)
    setattr(p, field, value)
    dummy = (ctypes.c_float * 4)()
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_init(p, ctypes.addressof(dummy))
    assert e.value.code == lib.AGENTS_EINVAL
    assert lib.agents_last_error(None)


def test_validation_rejects_bad_box(cdll):
    p = lib.agents_default_params(8, 8, 3, 2, 4)
    p.eps_lo[0] = 5.0
    p.eps_hi[0] = 1.0
    dummy = (ctypes.c_float * 4)()
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_init(p, ctypes.addressof(dummy))
    assert e.value.code == lib.AGENTS_EINVAL and "eps_lo" in str(e.value)


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="missing"):
        lib._lib_backup = None
        import importlib
        mod = importlib.import_module("paper_2510_16154_gb300._lib")
        saved = mod._lib
        try:
            mod._lib = None
            mod.load(str(tmp_path / "nope.so"))
        finally:
            mod._lib = saved


def test_warmstart_config_layout_and_validation(cdll):
    assert ctypes.sizeof(lib.ws_net_config) == 5 * 4 + 4 * 4
    cfg = lib.ws_net_config()
    cfg.in_ch, cfg.out_ch, cfg.base, cfg.levels, cfg.nsteps = 3, 6, 8, 1, 4   # levels < 2
    cfg.eps_lo[0] = cfg.eps_lo[1] = 2.0
    cfg.eps_hi[0] = cfg.eps_hi[1] = 1100.0
    h = ctypes.c_void_p()
    assert cdll.ws_net_create(ctypes.byref(cfg), None, ctypes.byref(h)) == lib.AGENTS_EINVAL
    assert b"invalid configuration" in cdll.ws_last_error()
    assert cdll.ws_conv3x3_forward(None, None, None, None, None, None, 1, 1, 1, 1, 1, 0, 0,
                                   None) == lib.AGENTS_EINVAL
    assert cdll.ws_conv3x3_backward_weight_workspace(2, 8, 8, 16, 32) > 0


def test_memory_limit_and_label_hook_without_a_device(cdll):
    # host-side state only: no context, no device call
    assert lib.agents_memory_held() == 0
    lib.agents_set_memory_limit(1 << 20)
    lib.agents_set_memory_limit(0)
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_debug_set_label_loop_cap(-5)
    assert e.value.code == lib.AGENTS_EINVAL
    lib.agents_debug_set_label_loop_cap(0)
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_debug_set_fused(1, -1, 0)
    assert e.value.code == lib.AGENTS_EINVAL
    with pytest.raises(lib.AgentsError) as e:
        lib.agents_debug_set_fused(5, 0, 0)
    assert e.value.code == lib.AGENTS_EINVAL
    lib.agents_debug_set_fused(0, 0, 0)
    lib.agents_debug_set_fused(1, 0, 0)
