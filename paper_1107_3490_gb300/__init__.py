"""GB300-native parallel-tempering Monte Carlo for the elastic bead-spring homopolymer.

The compute path is hand-written CUDA for sm_103a behind a C-ABI (``include/pt.h``);
``paper_1107_3490_gb300.pt`` is its thin ctypes binding and ``inputs`` makes seeded
synthetic inputs. Importing this package loads nothing; the binding loads the shared
library on first use and raises if it has not been built.
"""
__all__ = ["inputs", "pt"]
