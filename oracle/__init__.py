"""FP64 CPU oracle for SMS-MUSSELS -- TEST INFRASTRUCTURE, not product code.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path.

Parity status of each function (pins live in ``tests/test_oracle_pins.py``):

* fft2c / ifft2c ............ pinned (explicit DFT-matrix sums, unitarity)
* caipi_ramp ................ pinned (integer shift == circular image roll)
* forward / adjoint ......... pinned (dense DFT-matrix brute force at N=8,
                              adjoint dot test, A = I special case)
* hankel / hankel_adjoint ... pinned (entrywise definition, dot test; the
                              periodic variant likewise)
* gram ...................... pinned (trace closed form, PSD, rank bounds;
                              periodic: circular cross-correlation by FFTs)
* irls_weight ............... pinned (W^2 (G + eps I) = I)
* nullspace_weight .......... pinned (projector, annihilates a low-rank H)
* penalty ................... pinned (brute-force sum, W = I closed form,
                              periodic-FFT agreement on interior pixels;
                              periodic boundary: W = I and FFT agreement
                              at every pixel)
* cg ........................ pinned (exact solve in n steps, small SPD)
* sense ..................... pinned (least squares by a dense normal-equation
                              solve at N = 8; exact recovery of a phase-free
                              object)
* reconstruct ............... pinned (tests/test_oracle_solver_pins.py):
                              descent of the majorised Eq. 10 cost at fixed
                              eps; the fixed point is stationary for that
                              cost (finite differences of its eigenvalue
                              form); the last normal equations hold;
                              shot-permutation equivariance; noiseless
                              recovery (exact at lam = 0, first-order bias
                              of the penalty at lam > 0); slice- and
                              global-phase equivariance; each planted
                              mistake (weight exponent, dropped or halved
                              penalty, weight never updated) is caught
* magnitude ................. the root mean square over unit-phase shots returns rho
                              exactly (and squares average, not moduli)
"""
from .smsm_oracle import *  # noqa: F401,F403
from .smsm_oracle import (DEFAULT_PARAMS, adjoint, caipi_ramp, cg, fft2c, forward, gram,  # noqa: F401
                          hankel, hankel_adjoint, ifft2c, sense, irls_weight, magnitude, make_data,
                          normal, nrmse, nullspace_weight, penalty, reconstruct, shot_lines,
                          vdot)
