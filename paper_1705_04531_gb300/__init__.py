"""GB300-native inexact IETI-DP (MG-MG variant) for multipatch isogeometric
Poisson problems.

* ``workloads`` -- seeded synthetic problem descriptions (no arithmetic);
* ``build``     -- compiles ``libietidp.so`` (sm_103a) in-tree;
* ``ietidp``    -- ctypes binding of the C ABI (``include/ietidp.h``).

Importing the package does not load the CUDA library; ``import
paper_1705_04531_gb300.ietidp`` does, and fails if it has not been built.
"""
