"""FP64 CPU oracle for the differentiable charge+dipole particle-mesh Ewald.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its Python
binding) imports, links or executes anything in this package; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it. It shares
no code with the CUDA path; the only common dependency is the input generator module
``workloads``, which holds no method arithmetic.

Modules
-------
``bspline``  cardinal B-spline (Hockney-Eastwood) assignment weights W^(p) and their
             derivatives, Section 2.3.2 (Eq. w3d).
``ewald``    O1: explicit Ewald summation for point charges and point dipoles
             (real-space erfc images, reciprocal k-sum, self, neutralising background and
             surface terms) with analytic potentials, fields, field gradients and forces.
             Pinned by the rock-salt Madelung constant, alpha-independence, brute-force
             spherical image sums, translation invariance, zero net force and central
             finite differences.
``pme``      O2: plain particle-mesh Ewald written step by step as Section 2.3 states it
             (mesh, spline assignment with dipole derivative terms, FFT, deconvolved
             Gaussian-screened Green's function, energy), in float64 PyTorch CPU ops with
             autograd providing forces, dE/dq, dE/dmu and the Hessian-vector product of
             the force-matching backward, plus the erfc pair, self and background terms.
``meshdims`` the three mesh-size strategies of Section 2.3.1.

Parity status of each function is stated in its module header.
"""
