"""FP64 CPU oracle for the Lippmann-Schwinger forward model and its gradient.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or call anything in this package.  The CUDA library never routes through it
and shares no code, table or helper with it.

Everything here is plain numpy/scipy in float64/complex128, written from the
paper (arXiv 1910.13844) section by section:

* ``green``   -- scattering potential, Green function and the closed-form
                 spectrum of the truncated Green function (Sec. 2.1, Sec. 3.1,
                 eqs. GreenL / GreenL2), plus an independent radial quadrature.
* ``kernel``  -- the discrete Green operator of Theorem 1 (p-fold padding) and
                 the reduced-padding kernel of Proposition 1.
* ``model``   -- the discrete forward model (eqs. lipp1 / lipp2): matvec,
                 dense LU and BiCGStab solves, far field on the detector plane
                 (eq. Gtild-1), data-fidelity loss and its gradient (Alg. 1).
* ``mie``     -- scalar partial-wave solution for a homogeneous sphere, used as
                 a physics pin (Fig. 3 compares against such a solution).

Readings of the paper where it is silent, ambiguous or garbled:

* eq. GreenL: the sinc term is taken with a minus sign; with the printed plus
  sign the numerator does not vanish at ||w|| = k_b (a pole) and the value at
  0 disagrees with the integral of g over the ball.  sinc(x) = sin(x)/x.
* prefactor 1/(||w||^2 - k_b^2) as in eq. GreenL (Sec. 3.1 first line writes
  the opposite sign for the untruncated spectrum).
* truncation radius R = sqrt(Lx^2 + Ly^2 + Lz^2) (sqrt(3) L for a cube).
* DFT index sets are the centred sets [-N/2+1, N/2] of Sec. 1.4.
* the kernel value at the Nyquist offset d = n of the 2n grid never reaches a
  cropped output; it is set to zero.  The kernel is even in each axis (its
  spectrum too), so G is symmetric and G^H is the convolution with conj(K).
* far field G~: midpoint quadrature h^3 g(x_Gamma - z) of eq. Gtild-1.
* detector plane at x_Gamma = 3 L_z / 4 (top face of Omega at L_z/2),
  m x m pixels of pitch h centred on the optical axis.
* adjoint operator: (I - G^H diag f) (Sec. 4.2 prints diag(f) G~^*, which has
  incompatible dimensions).
* BiCGStab: x0 = u_in, stop on ||r|| <= tol ||b||, <a,b> = sum conj(a) b.
"""
