"""Seeded synthetic inputs for the GenEO-PCG solver (laminated hex blocks).

This package only builds input arrays: node coordinates, per-element material
ids and ply angles, the Dirichlet set, the load and the solver options.  It
holds none of the method's arithmetic, so both the FP64 CPU oracle and the CUDA
path consume exactly the same inputs without sharing any solver code.
"""
from .laminate import (PLY, RESIN, config, make_block, layer_cake,
                       CONFIG_NAMES, problem_summary)

__all__ = ["PLY", "RESIN", "config", "make_block", "layer_cake",
           "CONFIG_NAMES", "problem_summary"]
