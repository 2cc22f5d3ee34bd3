"""GB300-native coupled pseudopotential-flow + improved thermal lattice Boltzmann step.

The compute path is the CUDA library ``liblbpc`` (C ABI declared in ``include/lbpc.h``), built
for sm_103a by ``paper_1709_04400_gb300.build``. ``inputs`` holds the seeded synthetic inputs.
"""
