"""The oracle against the stored values under tests/golden/: values of the
paper's equations worked out by hand (each file cites the passage it
follows).  No GPU."""
import math
import os
from fractions import Fraction

import numpy as np

from oracle import drk_oracle as O
from paper_2412_11752_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def test_psi_values_of_eq9():
    rows = list(_rows("psi_eq9.txt"))
    assert len(rows) >= 20
    for tau, g, want in rows:
        tau, g, want = float(Fraction(tau)), float(Fraction(g)), float(Fraction(want))
        # the middle piece of Eq. 9 at tau = 0.99 has slope 199 and intercept
        # -99: its FP64 evaluation cancels about 100 x 2^-53 (1e-14)
        assert math.isclose(O.psi(g, tau), want, rel_tol=1e-13, abs_tol=1e-13), (tau, g, want, O.psi(g, tau))


def test_two_layer_worked_example_of_eq1():
    spec = {r[0]: r[1:] for r in _rows("two_layers_eq1.txt") if r[0] != "prim"}
    prims = [r[1:] for r in _rows("two_layers_eq1.txt") if r[0] == "prim"]
    w, h, fx, fy, cx, cy = (float(v) for v in spec["camera"])
    cam = synth.Camera(int(w), int(h), fx, fy, cx, cy)

    def field(p, key, n=1):
        i = p.index(key) + 1
        vals = [float(Fraction(v)) for v in p[i:i + n]]
        return vals if n > 1 else vals[0]

    f32 = lambda a: np.asarray(a, np.float32)
    K = 4
    sc = synth.Scene(
        mu=f32([[float(v) for v in p[:3]] for p in prims]),
        quat=f32([[1, 0, 0, 0]] * len(prims)),
        scale=f32([[field(p, "scale")] * K for p in prims]),
        theta=f32([[0, math.pi / 2, math.pi, 3 * math.pi / 2]] * len(prims)),
        eta=f32([field(p, "eta") for p in prims]),
        tau=f32([field(p, "tau") for p in prims]),
        opacity=f32([field(p, "opacity") for p in prims]),
        color=f32([field(p, "color", 3) for p in prims]),
        sh_degree=-1)
    bg = tuple(float(v) for v in spec["background"])
    px = np.array([[int(v) for v in spec["pixel"]]], np.int32)
    out = O.render_pixels(sc, cam, O.Options(bg=bg), px)
    rgb = [float(Fraction(v)) for v in spec["rgb"]]
    np.testing.assert_allclose(out["rgb"][0], rgb, atol=1e-12)
    assert math.isclose(out["T"][0], float(Fraction(spec["T"][0])), abs_tol=1e-12)
    assert out["n_contrib"][0] == len(prims)
