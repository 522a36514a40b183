"""Plain, slow, FP64 CPU oracle of the sketch-and-project ridge solver.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The
product library (``paper_2105_05565_gb300``) never imports, calls or links it,
and this package imports nothing from the product library.

What it computes follows the paper (arXiv 2105.05565, "RidgeSketch"):

* the ridge system A w = b in primal (A = X^T X + lambda I, b = X^T y) or dual
  (A = X X^T + lambda I, b = y, w = X^T alpha) form -- Section 2.1, eqs. (2)-(4);
* the sketch-and-project iteration -- Algorithm 1 (Section 3, update eq. (12),
  residual recursion eq. (13)) and its momentum form Algorithm 2 (Section 6.3,
  residual recursion eq. (53));
* the five sketches, each built as an explicit dense m x tau matrix S from its
  definition in Section 4 (Gaussian, Subsample, Count, SubCount, SRHT);
* the momentum parameter rules of Sections 6.1-6.2 and 8.1 (eqs. (38), (40),
  (49)-(50), (66), (67));
* importance-sampled coordinates p_j = A_jj / trace(A) and coordinate descent
  with momentum (``oracle.importance``, Section 7, eqs. (mSdisccolCD), (CDmom)),
  and the averaged iterates of the theorem of Section 5.2 (``average=True``);
* accelerated sketch-and-project (``oracle.accel``, Algorithm 3 of Section 9);
* kernel ridge regression with the RBF kernel (``oracle.kernel``, Section 2.2);
* Conjugate Gradients on the same system (``oracle.cg``, the competitor of
  Section 8.3);
* the learned sketch proposal (``oracle.learned``): features, the scoring
  network and its gradient, the proposal, Gumbel-top-tau selection, the
  per-coordinate labels from the projection identity of Section 3, and Adam.

Random choices come from the counter-based generator in ``oracle.rng`` which is
written from the published SplitMix64 definition; the GPU library implements
the same generator separately, so that sketch indices and signs agree bit for
bit without sharing code.

Parity status of each function is stated in its docstring ("pinned by ...").
"""
from .rng import (  # noqa: F401
    GAMMA,
    mix64,
    draw,
    iter_key,
    sample_keys,
    subsample_indices,
    signs_buckets,
    gaussian_entries,
)
from .sketches import sketch_matrix, subcount_params, default_tau  # noqa: F401
from .momentum import momentum_schedule  # noqa: F401
from .solver import (  # noqa: F401
    form_system,
    direct_solution,
    least_norm_solution,
    sketch_and_project,
    solve_ridge,
    solve_matrix_free,
    true_residual,
)
from . import learned  # noqa: F401,E402
from . import importance  # noqa: F401,E402
from . import cg  # noqa: F401,E402
from . import accel  # noqa: F401,E402
from . import kernel  # noqa: F401,E402
