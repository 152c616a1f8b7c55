"""FP64 CPU oracle for the Adaptive-FAM micro-model hot path (arxiv 2409.00184).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it. It shares no code, headers,
tables or constants with the CUDA library; both sides only receive the same seeded
inputs from ``synth``.

What each module computes, and the passage it follows:

* ``bspline``  - clamped knot spans and the Cox-de Boor recurrence for N_{i,p} and
  N'_{i,p}. The paper uses B-spline micro-models (MFA, Sec. 4.2 and the "geometric
  bases" of Sec. 1) without writing the basis out; the oracle uses the textbook
  definition (de Boor's recurrence; span finding as in Piegl & Tiller A2.1).
* ``decode``   - value and parametric gradient of the trivariate tensor-product
  model f(u,v,w) = sum N_a(u) N_b(v) N_c(w) P_abc, evaluated directly per point
  over the (p+1)^3 nonzero terms (the queries valueMicroModel / gradientMicroModel
  of Algorithm 4).
* ``encode``   - least-squares fit of control points to the n^3 samples of a
  micro-block (the model(NCP, degree) call of Algorithm 1) and its RMSE error
  (Table 1's error metric); Eq. 2 model size; Eq. 4 NCP* selection.
* ``adjoint``  - dP = sum_s r_s N_a(u_s) N_b(v_s) N_c(w_s), the gradient of
  0.5*||decode(P) - D||^2 with respect to P.
* ``raycast``  - front-to-back direct volume rendering with early termination
  (Algorithm 4) over a bricked value+gradient cache.
* ``multires`` - shared-boundary micro-blocks of every level of detail (Sec. 4.2),
  the selection of a level per block by the distance from the point of view
  (Sec. 5.1.3), Algorithm 4 over the selected models, and the MSE / PSNR image
  metrics of Sec. 5.2.

Parity pins (tests/test_oracle_*.py) tie every function to something other than
itself: partition of unity, Bernstein closed forms, polynomial reproduction, endpoint
interpolation, finite differences, brute-force dense least squares, the adjoint
dot-product identity, and for the ray caster closed forms of each of its steps (camera
orientation and centre ray, chord length and sample positions, front-to-back sums,
termination, opacity correction, transfer-function interpolation, shading, trilinear
interpolation across bricks). The renderer's choices that the paper leaves open (camera
model, lighting model, sampling rate) are readings stated in oracle/raycast.py; the pins
fix the oracle to those readings, not the readings to the paper.
"""

from . import bspline, decode, encode, adjoint, raycast, multires  # noqa: F401
