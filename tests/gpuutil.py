"""Helpers for the GPU parity tests: build/load the C-ABI library, move arrays, and
build matching parameter sets for the library and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2510_16154_gb300 import lib            # noqa: E402
from paper_2510_16154_gb300.build import build     # noqa: E402
import oracle                                      # noqa: E402

_built = False


def ensure_lib():
    global _built
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not _built:
        build()
        lib.load()
        _built = True


def dev(a, dtype=None):
    a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))
    return torch.from_numpy(a).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def params(H, W, C, R, T, **kw):
    """(library params, oracle Params) for the same problem."""
    p = lib.agents_default_params(H, W, C, R, T)
    for k, v in kw.items():
        if k in ("eps_lo", "eps_hi"):
            getattr(p, k)[0], getattr(p, k)[1] = v
        else:
            setattr(p, k, v)
    op = oracle.Params(radius=R, nsteps=T, dt=p.dt, alpha=p.alpha, rho=p.rho, gamma=p.gamma,
                       eps_lo=(p.eps_lo[0], p.eps_lo[1]), eps_hi=(p.eps_hi[0], p.eps_hi[1]),
                       norm_mode=p.norm_mode, tv_mode=p.tv_mode)
    return p, op


def f32(a):
    """Round to float32 and back: the exact values the GPU stores."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def zeros_dev(*shape, dtype=None):
    return torch.zeros(*shape, dtype=dtype or torch.float32, device="cuda")


def assert_control_derivative(D, Dw, rel=1e-5, negligible=1e-6):
    """D = (D_x, D_c) per step against the oracle's, each component against its OWN
    largest entry (relative rel).  Only a component below `negligible` times the other's
    largest entry (truly negligible: far below what float32 resolves beside it) is
    checked against rel times the largest entry of D instead."""
    D = np.asarray(D, dtype=np.float64).reshape(-1, 2)
    Dw = np.asarray(Dw, dtype=np.float64).reshape(-1, 2)
    top = float(np.max(np.abs(Dw)))
    assert top > 0
    for k, name in ((0, "D_x"), (1, "D_c")):
        m = float(np.max(np.abs(Dw[:, k])))
        scale = m if m >= negligible * top else top
        err = float(np.max(np.abs(D[:, k] - Dw[:, k])))
        assert err <= rel * scale, (name, err, m, top)
