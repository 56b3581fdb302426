"""Plain, slow FP64 / complex128 CPU oracle of the RBM-VMC + SR method.

TEST INFRASTRUCTURE ONLY.  Nothing in the library path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA path; both sides read the same seeded inputs from
``paper_1904_00031_gb300.workloads`` (problem definitions only).

Modules and the passages of the NetKet paper (arXiv:1904.00031) they follow:

* ``philox``    Philox4x32-10 counter-based generator (Salmon et al., SC'11);
                the paper names Metropolis sampling (Sec. 2.2.5) but no generator.
* ``rbm``       RBM amplitude psi(sigma) = exp(a.sigma) prod_j cosh(theta_j),
                theta = W sigma + b (Sec. 2.2.2, RbmSpin; lncosh form of the
                single-layer FFNN, Sec. 2.2.2) and its analytic log-derivatives
                (Sec. 2.2.5).
* ``hamiltonian`` Sparse matrix of a GraphOperator-style Hamiltonian, full ED and
                Lanczos (Sec. 2.1, ``exact`` module), the TFIM free-fermion closed form.
* ``rbm_symm``  symmetric RBM (RbmSpinSymm, Sec. 2.2.2): tied weights over a lattice
                symmetry group, its tied log-derivatives, and SR in the tied space.
* ``ffnn``      multi-layer feed-forward network of dense layers and ln cosh
                activations with a sum output (Sec. 2.2.2, FFNN), its holomorphic
                log-derivatives and backward.
* ``local_energy`` E_loc(sigma) = sum_sigma' H_{sigma sigma'} psi(sigma')/psi(sigma)
                (the energy estimator equation of Sec. 2.2.5).
* ``sampler``   Metropolis Markov chains over |psi|^2 with single-spin-flip and
                nearest-neighbour exchange moves (Sec. 2.2.5; listing of Sec. 3.1).
* ``tempering`` parallel tempering (replica exchange) of Metropolis chains over
                |psi|^(2 beta) ladders (the sampler option named in Sec. 2.2.5).
* ``supervised`` the negative log overlap loss of Eq. 1 (Sec. 2.2.3), its gradient
                from samples of the target, and AdaMax (Kingma and Ba, Algorithm 2).
* ``sr``        energy statistics, the SR system S delta = F solved exactly or by
                conjugate gradient, and the SGD step alpha <- alpha - lambda delta
                (Sec. 2.2.5; Eq. (2) of Sec. 2.2.3).
* ``vmc``       one full VMC + SR iteration in the paper's order (Sec. 2.2.5).

Readings of passages where the paper is silent are listed in each module.
"""
