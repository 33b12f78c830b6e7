"""FP64 CPU oracle of the wavelet-domain MAP tomography solve (Helin & Yudytskiy,
"Wavelet methods in multi-conjugate adaptive optics", Secs. 2-5).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports, links or
calls it, and this package imports nothing from the product; the two share only
the seeded input generators in ``synth``.

It is a plain, slow, obviously correct restatement of the paper's definitions
in numpy float64, in the paper's order and notation:

* ``wavelets``    - orthonormal Daubechies filters, periodic 2-D pyramid W, W^-1;
* ``atmosphere``  - NGS/LGS ray-tracing P (with the cone effect) and its
                     transpose, Fried-geometry Shack-Hartmann slopes Gamma and
                     its transpose;
* ``tomography``  - noise weighting with tip/tilt removal, diagonal wavelet prior
                     D, the normal operator of eq. eqn_lse, its right-hand side,
                     the modified Jacobi diagonal, and Hestenes-Stiefel (P)CG;
* ``fitting``     - the fitting step: piecewise-bilinear mirrors H, the NGS
                     projections P over the evaluation directions, CG on
                     H^T H a = H^T P phi, and the Marechal Strehl of a correction;
* ``control``     - pseudo-open-loop control: the mirrors measured by the
                     sensors (A_hat) and one step of the two-frame-delay loop.

Each function is pinned by tests/test_oracle_*.py against closed forms,
invariants, textbook special cases and brute force on tiny inputs; nothing in
those pins comes from the CUDA path.
"""
from .tomography import Tomography
from .fitting import Fitting
from .control import Control
from . import wavelets, atmosphere, tomography, fitting, control

__all__ = ["Tomography", "Fitting", "Control", "wavelets", "atmosphere", "tomography", "fitting", "control"]
