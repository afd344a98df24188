"""Plain CPU oracle of the 2D electromagnetic PIC step (Guidotti 2021, §3.1-3.2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library (``paper_2501_14795_gb300``) never imports it and
shares no code with it.

Parity status per function (what pins each one; the pins live in
``tests/test_oracle_*.py``):

* ``orc_gather``   pinned: uniform and linear fields are reproduced exactly at
  every staggered location; brute-force bilinear sums on random fields.
* ``orc_boris``    pinned: |u| kept exactly in a pure B field; gyration angle
  2 atan(|q/m| B dt / 2 gamma) per step; pure-E closed form u0 + (q/m) E t.
* ``orc_deposit_move`` pinned: discrete continuity (Eq. 12) to round-off for
  same-cell, 4-, 7- and 10-boundary moves; additivity under sub-division of the
  move; total current equal to q v; Jz weights summing to one.
* ``orc_advance``  pinned through the gyration orbit, cold-plasma oscillation
  frequency, two-stream growth rate and Gauss-law invariance.
* ``orc_yee``      pinned: vacuum plane-wave frequency against the Yee
  dispersion relation; div B kept at zero.
* ``orc_rho``      pinned: the weights of each particle sum to its charge; a
  uniform lattice gives a uniform density.
* ``orc_tile_sort`` pinned: equal to numpy's stable argsort by tile id.
* ``tile_order`` / ``tile_offsets_in_order`` (the order of the tiles in the
  arrays: rows, or with the moving window columns from the right edge) pinned
  by brute-force counts of the particles in each tile of that order.
* ``binomial_filter`` pinned: the closed-form response cos^2(k dx/2) cos^2(k dy/2)
  per pass on single Fourier modes, exact conservation of the sum (k = 0), the
  Nyquist mode removed, brute-force 3x3 stencil (1 2 1)(1 2 1)/16.
* Weibel growth (config with counter-streaming populations along z): parity
  only bounded, between 0.7x and 1x the cold-fluid rate (the thermal spread
  lowers the cold rate by an amount the thesis does not give).
* ``window`` (module: moving window, injection, lasers; readings in its
  docstring): the window position pinned against exact rational arithmetic;
  shift, removal and injection together pinned by the exact invariance of a
  cold plasma at rest (with a part-filled edge column); the open box's
  dropped current by additivity; the plane pulse by the Yee scheme's own group
  velocity and energy conservation (fixed box and moving window); the Gaussian
  beam by its diffraction down to the waist at the focus; the polarisation by
  the rotated pulse and B = x_hat x E.
* ``denoiser`` (module): circular 3x3 convolution pinned by brute force and an
  FFT correlation; its input, weight and bias gradients by adjoint identities
  and brute force; pooling / upsampling adjoints; the whole network's gradient
  by central finite differences; Adam by its first step and convergence on a
  quadratic; bfloat16 rounding by hand-computed bit patterns.
"""
from .oracle import (  # noqa: F401
    OracleSim,
    SpeciesState,
    build_oracle,
    lib,
    gather,
    boris,
    deposit_move,
    advance,
    yee,
    binomial_filter,
    rho_nodes,
    tile_sort,
    tile_order,
    tile_offsets_in_order,
    field_energy,
    div_e,
    div_j,
    ORC_EPARTICLE,
)
