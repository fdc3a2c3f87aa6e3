"""Float64 CPU oracle for the randomized range finder / randomized SVD.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``; the
library (``paper_1607_01649_gb300``) never does, and the two share no code.

Parity status per function:
* philox4x32_10 / gaussian: pinned (independent Philox implementation,
  distribution tests, prefix property).
* orth, rsvd_basic, rsvd_power, rsvd_power_plain, stage_b: pinned (exact
  recovery of rank-k matrices, full SVD when l = min(m, n), Stage-B identity,
  singular-value interlacing, Eckart-Young, expectation/tail/power bounds,
  the A^(q) closed form, round-off ablation).
* adaptive_blocked, single_vector_range_finder, adaptive_range_finder:
  pinned (Frobenius identity of Sec. 12.4, residual <= eps, rank vs the
  eps-rank from a full SVD, span equivalence with the block method).
* certificate, spectral_residual: pinned (eq. (infomm), Lemma
  thm:aposteriori statistically, direct 2-norm on small cases).
* controller (probe features, MLP forward / loss / gradient, Adam step,
  decision rule, labels from the adaptive ranks, residual estimate): pinned
  (sigma(Q G) = sigma(G) through eigvalsh, scale invariance, hand-built
  networks, uniform-logit loss, central finite differences, the closed-form
  first Adam step, brute-force label and eps-rank checks, eq. (infomm) and
  Lemma thm:aposteriori over seeds).  What the trained network predicts has
  no pin: it is judged by the gain it brings, not by parity.
* fp8 (e4m3 values, rounding, row/column scaling, the scaled sketch
  products): pinned (the value set and all 256 codes from the format's
  definition, round trip, ties to even at every midpoint, saturation, brute
  force over 8000 values, exact products on representable operands).
* nystrom (Fig. nystrom): pinned (exact recovery when rank(A) = k + p, the
  Loewner order F F* <= A, the closed form A^1/2 (I - P) A^1/2 of the
  residual, the explicit-inverse form of eq. spd_nystrom, the accuracy gain
  over eq. spd_standard across seeds).
* singlepass_evd, singlepass_svd (Figs. singlepass_herm, singlepass_gen):
  pinned (exact recovery of rank-k inputs with C = Q* A Q, both
  least-squares fits against their stationarity conditions solved as
  Sylvester equations, the free / constrained / symmetrized fit ordering,
  the section's loss of accuracy against two passes).  No GPU path yet.
* srft_omega, rsvd_srft (eq. SRFT): pinned (orthonormal columns, numpy's FFT
  as the subsampled transform, uniformity of D and S, prefix property, exact
  recovery, accuracy near the Gaussian sketch).  No GPU path yet.
* rsvd_block_krylov (Sec. "Extended sampling matrix"): pinned (q = 1 is
  Fig. RSVD, exact recovery of rank q l, span of a blockwise orthonormalized
  Krylov basis, residual below the power scheme's by nesting).  No GPU path yet.
* adaptive_blocked_spectral (the blocked scheme with Fig. adaptive2's
  spectral stopping test, the GPU form planned for that row): pinned (the
  blocked scheme's basis bit for bit, spectral error below eps on every seed,
  rank between the spectral eps-rank and the Frobenius rank at a quarter of
  the threshold plus two blocks).  No GPU path yet.
* rsvd_power_centred (implicit column centring for PCA): pinned (equals the
  fixed-rank oracle on the explicitly centred matrix; 1* U = 0).  No GPU path yet.
"""
from .philox import (philox4x32_10, gaussian, omega_words, box_muller, seed_key,
                     STREAM_SKETCH, STREAM_ADAPTIVE, STREAM_CERTIFY, STREAM_ADAPTIVE2, STREAM_NORM,
                     STREAM_ROW, STREAM_SRFT_D, STREAM_SRFT_S)
from .rsvd import orth, sign_normalize, stage_b, rsvd_basic, rsvd_power, rsvd_power_plain
from .norms import fro_residual, spectral_residual, certificate, theorem_bounds
from .adaptive import (adaptive_blocked, adaptive_blocked_spectral, truncate_to_tol,
                       single_vector_range_finder, adaptive_range_finder)
from . import controller
from . import fp8
from .nystrom import nystrom
from .singlepass import singlepass_evd, singlepass_svd
from .srft import srft_omega, rsvd_srft
from .krylov import rsvd_block_krylov
from .centred import rsvd_power_centred
