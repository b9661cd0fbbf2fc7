"""GB300 (sm_103a) implementation of the Simplex-GP permutohedral-lattice kernel MVM and
the batched conjugate-gradient solve that drives it (Kapoor et al., 2021, Sec. 3-4).

The compute path is libsgp.so (CUDA kernels behind the C-ABI of include/sgp.h); this
package only marshals arguments to it.
"""

from ._lib import SGPError  # noqa: F401


def __getattr__(name):
    if name in ("Lattice", "lattice_mvm", "trim_memory"):
        from . import lattice

        return getattr(lattice, name)
    raise AttributeError(name)
