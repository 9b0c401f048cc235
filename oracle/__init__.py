"""FP64 CPU oracle for the affine reconstructed nodal DG (aRDG) method (Song & Srinivasan,
arXiv 1912.06221).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only the test
suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs call it.
It is a plain, slow, step-by-step NumPy/SciPy restatement of the method in the paper's
order and notation, sharing no code with the CUDA library (the seeded input generators in
``synth`` are the only common module and hold none of the method's arithmetic).

Modules
  refops   reference-element operators (Sec. 3), node reorderings (Sec. 4.4),
           reconstruction system (Sec. 4.5)
  mesh     connectivity, periodic matching, affine geometry (Eqs. mapping_tri,
           triangle_jacobian)
  ardg     enclosed parallelogram (Sec. 4.2), projections (Eq. totalProjection),
           reconstruction and edge gradient (Algorithm aRDG), D reconstruction (Algorithm 2)
  rhs      semi-discrete right-hand side (Eq. NDG_diffusion_once_matrixForm_Fullyreference
           with the convective flux of Eq. convection_diffusion), SSP-RK3, error norms
           (Eqs. L2_norm_cellUnit, Linf_norm_cellUnit), dense operator
"""
