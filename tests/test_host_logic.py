"""CPU checks of host-side logic of the package: the warm-start network's flat parameter
layout agrees with the oracle's for every configuration the library accepts, the
committed weights file matches its own specification, and the high-resolution transfer
scales the window radius as documented (round(factor R), at least 1), and the warm
start's lift factor brings an image to the training resolution (256) by powers of two
that divide both sides."""
import json
import os

import numpy as np
import pytest

from oracle import cnn
from paper_2510_16154_gb300.hires import transfer_radius
from paper_2510_16154_gb300.warmstart import NetSpec, WEIGHTS_DIR, lift_factor


@pytest.mark.parametrize("levels", [2, 3, 4, 5, 8])
@pytest.mark.parametrize("base,in_ch,out_ch,T", [(8, 3, 6, 4), (32, 3, 6, 20), (16, 31, 62, 7)])
def test_parameter_layout_matches_oracle(levels, base, in_ch, out_ch, T):
    spec = NetSpec(in_ch=in_ch, out_ch=out_ch, base=base, levels=levels, nsteps=T)
    cfg = cnn.NetConfig(in_ch=in_ch, out_ch=out_ch, base=base, levels=levels, nsteps=T)
    assert spec.param_shapes() == cnn.param_shapes(cfg)
    names = [n for n, _ in spec.param_shapes()]
    assert len(names) == len(set(names))
    # encoder, decoder and head convolutions, then the control head
    assert len(names) == 2 * (2 * levels + 2 * (levels - 1) + 1) + 2


def test_committed_weights_match_their_spec():
    path = os.path.join(WEIGHTS_DIR, "warmstart_rgb_T20_R5.npz")
    z = np.load(path)
    d = json.loads(str(z["spec"]))
    d["eps_lo"], d["eps_hi"] = tuple(d["eps_lo"]), tuple(d["eps_hi"])
    spec = NetSpec(**d)
    theta = z["theta"]
    assert theta.dtype == np.float32 and theta.ndim == 1
    assert theta.size == sum(int(np.prod(s)) for _, s in spec.param_shapes())
    assert np.all(np.isfinite(theta))
    assert (spec.in_ch, spec.out_ch, spec.base, spec.levels) == (3, 6, 32, 4)


@pytest.mark.parametrize("radius,factor,want", [(5, 2.0, 10), (5, 1.0, 5), (2, 0.5, 1),
                                                (1, 0.25, 1), (3, 1.5, 4), (7, 4.0, 28)])
def test_transfer_radius(radius, factor, want):
    assert transfer_radius(radius, factor) == want


@pytest.mark.parametrize("H,W,f", [(256, 256, 1), (2048, 2048, 8), (1024, 512, 2),
                                   (2048, 1536, 4), (1100, 1100, 4), (600, 600, 2),
                                   (64, 64, 1), (512, 768, 2)])
def test_lift_factor(H, W, f):
    assert lift_factor(H, W) == f
    assert H % f == 0 and W % f == 0 and min(H, W) // f >= min(256, min(H, W))
