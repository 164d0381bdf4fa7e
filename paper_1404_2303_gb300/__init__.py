"""GB300-native SPH neighbour interactions over sorted cell pairs.

Python surface of libsphgb.so: ``SPH`` (context: build, density with the
smoothing-length solve, force, adjoints) and ``SPHDensityForce`` (a
torch.autograd.Function).  PyTorch provides device memory and streams only;
every step runs in the CUDA library.
"""
from .sph import SPH, default_params  # noqa: F401
from .autograd import SPHDensityForce, sph_density_force  # noqa: F401
