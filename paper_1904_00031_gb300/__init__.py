"""GB300-native (sm_103a) RBM variational Monte Carlo + stochastic reconfiguration,
after NetKet (Carleo et al., arXiv:1904.00031).

* ``nk``        thin binding of the C ABI declared in ``include/nk.h``
* ``vmc``       one VMC + SR iteration driven through the C ABI
* ``workloads`` seeded synthetic inputs (lattices, operators, parameters)
* ``build``     compiles ``csrc/*.cu`` into ``libnk.so`` for sm_103a

Importing the package loads nothing; the library is loaded on first use.
"""
