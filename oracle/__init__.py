"""Plain FP64 CPU oracle for the FC-DOM time march of the 2D time-domain
radiative transfer equation (Gaggioli & Bruno, arXiv 2202.09421).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may
import it. The product path (the CUDA library and its binding) never imports,
links or executes anything here, and nothing here imports the product.

Every function restates the paper's method in its own order and notation:

* Sec. 2, eq. (Toper)/(RTE): transport operator, Fresnel boundary condition;
  eq. (Henyey-Greenstein) phase function; eq. (sourcelabwind) window.
* Sec. 3.1, eqs. (RTEsources), (OpMed), (FObj): beams, detectors, objective.
* Sec. 3.4, eq. (AdjointProblem), eq. (gradient_fin); Sec. 3.6 eq. (FDwin22).
* Sec. 4.1 eq. (RTETrapz): discrete ordinates and trapezoid weights, phase
  normalisation; Sec. 4.2 eqs. (RTEAB4)/(RTEAB4L): Adams-Bashforth 4;
  Sec. 4.3 eqs. (RTEFCSum), (FFilter), (RTEFCSumder): FC-Gram continuation
  and the filtered spectral derivative; Algorithm 1: loop order.
* Sec. 4.4 / Algorithm 1: the subdomain decomposition with two fringe
  points (fcgram.fc_derivative_parts, Solver(fc_parts=...)).
* The exact discrete adjoint and the tangent-linear march of the discrete
  scheme (Solver.discrete_adjoint_gradient, tangent_linear_objective): the
  transpose of eqs. (RTEAB4)/(RTE)/(OpMed)/(FObj) as discretised, an
  extension of Sec. 3.4 pinned by the dot-product identity, central
  differences and a dense brute-force sensitivity on a tiny grid.

Floating point is FP64 throughout; numpy's FFT serves as the FFT step.
"""
