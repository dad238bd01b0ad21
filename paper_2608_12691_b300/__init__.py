"""B300-native alchemical nonbonded engine for lambda-dynamics (linear-basis-
function coupling, Ewald/PME Coulomb, capped soft-LJ basis, dual OPES on the
mirror-periodic alchemical coordinate).

The computation lives in the CUDA library ``liblfe.so`` (C-ABI in
``include/lfe.h``); ``paper_2608_12691_b300.lfe`` is its ctypes binding and
``paper_2608_12691_b300.systems`` builds the seeded synthetic inputs.
"""
