"""FP64 CPU oracle for the batched self-energy integrand (test infrastructure).

This package is a plain, slow, diagram-by-diagram restatement of what the GPU
path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product library never does.
It shares no code with ``paper_2403_18840_gb300``: the only common module is
``workloads`` (seeded workload descriptions, no arithmetic of the method).

Modules
-------
philox       Philox4x32-10 counter-based generator (Salmon et al., SC'11)
conventions  units and UEG parameters (Sec. VI.A, Eq. ueg_action)
diagrams     brute-force enumeration of self-energy topologies (Sec. II.A)
leaves       G0 and V with their counterterm derivatives (Eqs. propagator,
             green_ct, interaction_ct)
integrand    hypercube map and per-sample integrand roots Sigma^(n,m,l)
             (Eqs. sigma_integration, sigma_xi_dmu_dlambda)
vegas        VEGAS separable map, histogram and grid update (Sec. IV)
flow         affine coupling flow: sample, density, forward-KL loss and
             gradient (Appendix A, Eqs. NFtransform, coupling_layer)
postprocess  counterterm post-processing and m*/m (Sec. VI.A, Eqs.
             counterterm, eff_mass_ratio, dsigma_depsilon_series)

Parity status of each function is stated in its docstring; functions with no
independent pin say "parity unpinned".
"""
