"""FP64 CPU oracle for the directional SLSHT (Khalid et al., arXiv:1207.5558).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference leg of
``bench.py``, and by nothing else.  The CUDA library never imports, links or
calls it, and it shares no code with the CUDA path: the only module both sides
use is ``synth`` (seeded synthetic inputs, none of the transform's arithmetic).

Everything here is plain numpy in float64 (plus exact rational arithmetic for
the Wigner-3j pins), written to be read against the paper, not to be fast.

Modules
  special  spherical harmonics (Eq. Sph_harmonics), Wigner d by its textbook
           three-term recurrence in the degree, exact Wigner-3j (Racah formula),
           Gaunt coefficients (the triple product T of Sec. III-B).
  slsht    the transform: modulated-signal coefficients (Appendix A,
           Eq. sht_sep_variable), the forward distribution by direct quadrature of
           the definition (Eq. stft_spatial) and by the convolution form
           (Eq. alternative_harmonic_formulation_wigner), the SO(3) quadrature
           weights and the inverse (Eq. inversion_1, inversion_2,
           sig_reconstruction_discrete), and the inverse without h_0^0 of the
           remark after Eq. inversion_2 (projection on conj(D^p_{q,q'}) and
           the Wigner-3j orthogonality).
  window   the elliptical concentration window of Sec. III-D (Eq. region_def
           and the concentration matrix), the reference of the device window
           generator and the source of the stored windows of workloads 2, 5.

Parity status of every function is stated in its docstring: each one is pinned
by a ``-m "not gpu"`` test against something other than itself (closed forms,
exact rationals, library routines, invariants the paper states).
"""

from . import special, slsht, window  # noqa: F401
