"""Writes the stored concentration windows of workloads 2 and 5:
workload2_window.json (L_h = 8, the 20 x 10 degree ellipse) and
workload5_window.json (L_h = 64, the 8 x 3 degree ellipse), each the most
concentrated band-limited eigenfunction of its elliptical region
(Sec. III-D, Eq. region_def), computed by the oracle (oracle/window.py).

They are test INPUTS: the seeded-input module reads them so that neither the
tests nor the benchmark spend a minute on the 4096 x 4096 concentration
eigenproblem of workload 5, and the device window generator is checked
against them.  The semi-axes become (theta_c, a) by cos a = cos theta_c cos b
(spherical Pythagoras for an ellipse centred on the pole).  This script
imports only the oracle and numpy.  Regenerate with
`python tests/golden/make_windows.py`."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.window import window_ellipse  # noqa: E402

WINDOWS = {2: (8, (20.0, 10.0)), 5: (64, (8.0, 3.0))}


def focus_from_axes(a_deg, b_deg):
    a, b = np.deg2rad(a_deg), np.deg2rad(b_deg)
    return float(np.arccos(np.cos(a) / np.cos(b))), float(a)


def main():
    for w, (L, axes) in WINDOWS.items():
        h, lam = window_ellipse(L, *focus_from_axes(*axes))
        out = {"_about": f"workload {w} window: L_h = {L} concentration eigenfunction of the "
                         f"{axes[0]:g} x {axes[1]:g} degree ellipse (Sec. III-D), flat index p*p+p+q; "
                         "written by tests/golden/make_windows.py from oracle/window.py",
               "Lh": L, "axes_deg": list(axes), "concentration": lam,
               "re": [float(v) for v in h.real], "im": [float(v) for v in h.imag]}
        with open(os.path.join(HERE, f"workload{w}_window.json"), "w") as fh:
            json.dump(out, fh)


if __name__ == "__main__":
    main()
