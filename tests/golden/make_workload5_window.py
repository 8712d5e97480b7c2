"""Writes workload5_window.json: the L_h = 64 window of workload 5, the most
concentrated band-limited eigenfunction of the 8 x 3 degree elliptical region
(Sec. III-D, Eq. region_def), as synth/window.py draws it.

It is a test INPUT, not an expected value: stored so the workload-5 GPU test
does not spend a minute on the 4096 x 4096 concentration eigenproblem each
run.  Regenerate with `python tests/golden/make_workload5_window.py`."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synth.window import ellipse_from_axes, window_ellipse  # noqa: E402


def main():
    h = window_ellipse(64, *ellipse_from_axes(8.0, 3.0))[0]
    out = {"_about": "workload 5 window: L_h = 64 concentration eigenfunction of the 8 x 3 degree ellipse "
                     "(Sec. III-D), flat index p*p+p+q; written by make_workload5_window.py from synth/window.py",
           "Lh": 64, "axes_deg": [8.0, 3.0],
           "re": [float(v) for v in h.real], "im": [float(v) for v in h.imag]}
    with open(os.path.join(HERE, "workload5_window.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
