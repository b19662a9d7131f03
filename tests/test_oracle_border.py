"""The absorbing border (the stand-in for the paper's PML, an Im n^2 layer of the
workload recipe) as the oracle propagates through it, pinned by physics rather
than by the oracle itself:

- Im n^2 >= 0 makes the medium passive, so no step may raise the field's L2 norm;
- a beam tilted 20 degrees towards the border loses most of its energy once it
  has crossed the border;
- what comes back (energy in the kx < 0 half of the spectrum, where the beam has
  almost none) stays at the percent level.

A border with the wrong sign (gain) fails the first check, a missing one the
second, a hard-edged one the third."""
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _march(sign=1.0, steps=24):
    from oracle import aaa_lawson, operators as ops, propagator as orp
    from paper_2410_17446_gb300 import workloads as wl
    with open(os.path.join(ROOT, "paper_2410_17446_gb300", "tables", "plain_scalar_64.json")) as f:
        T = aaa_lawson.PoleTable.from_json(json.load(f))   # dz = lambda/2 at dx = lambda/8
    g = wl.Grid(64, 64, 1 / 8, 1 / 8)
    n2 = 1.0 + sign * 1j * wl.absorbing_sigma(g, 8, 0.2)
    X, _ = g.mesh()
    w = (wl.gaussian_beam(g, 1.0) * np.exp(1j * 2 * math.pi * math.sin(math.radians(20)) * X))[None]
    med = ops.Medium(n2, g.dx, g.dy, 2 * math.pi, 1.0, 1)
    kx = np.fft.fftfreq(g.nx, g.dx)
    E0 = float(np.sum(np.abs(w) ** 2))
    energy, back = [1.0], []
    F = np.fft.fft2(w[0])
    back0 = float(np.sum(np.abs(F[:, kx < 0]) ** 2) / F.size) / E0
    for _ in range(steps):
        w, _st = orp.step(med, w, T, tol=1e-11)
        energy.append(float(np.sum(np.abs(w) ** 2)) / E0)
        F = np.fft.fft2(w[0])
        back.append(float(np.sum(np.abs(F[:, kx < 0]) ** 2) / F.size) / E0)
    return np.array(energy), np.array(back), back0


def test_border_is_passive_absorbing_and_reflects_little():
    energy, back, back0 = _march()
    assert np.all(np.diff(energy) <= 1e-9), energy          # passive: the norm never grows
    assert energy[-1] < 0.5, energy[-1]                      # the crossing beam is absorbed
    assert back.max() - back0 < 0.02, (back0, back.max())    # little comes back


def test_border_with_gain_would_fail_the_pin():
    """The same march with the border's sign flipped (a gain layer) raises the norm."""
    energy, _, _ = _march(sign=-1.0, steps=12)
    assert energy[-1] > 1.0
