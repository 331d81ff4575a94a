"""Walk on stars (Sawhney et al. 2023) on GB300: a CUDA walk megakernel over a
BVH (Dirichlet) and a spatialized normal-cone hierarchy (Neumann), behind the
C ABI declared in include/wost.h.

Importing the package loads nothing native; ``paper_2302_11815_gb300.wost``
loads the CUDA library on first use and raises if it is missing.
"""
