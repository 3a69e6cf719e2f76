"""Seeded synthetic input grids shared by the CUDA library's tests/bench and the
oracle's tests.

This package builds input *data* only (tree topology, per-leaf dust opacity and
stellar emissivity, dust albedo and Henyey-Greenstein g, point sources).  It
holds none of the radiative-transfer arithmetic: no ray tracing, no HEALPix, no
phase function.  Every geometric value it emits is exactly representable in
float32 so that the float32 GPU path and the float64 oracle see bit-identical
inputs.
"""
from .grids import (Grid, lattice_grid, refine_tree, sphere_cube, galaxy_disk,
                    lognormal_cube, config1, config2, small_sphere, galaxy_particles, particle_galaxy,
                    config5)

__all__ = ["Grid", "lattice_grid", "refine_tree", "sphere_cube", "galaxy_disk",
           "lognormal_cube", "config1", "config2", "small_sphere",
           "galaxy_particles", "particle_galaxy", "config5"]
