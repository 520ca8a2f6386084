"""Seeded synthetic inputs shared by the oracle and the GPU path.

This package holds only input generators: the jittered Kuhn tetrahedral mesh
family (6 tetrahedra per hexahedron), its regular periodic variant, and closed-form
velocity fields used as initial and Dirichlet boundary data.  It contains none of the discretisation's
arithmetic (no bases, quadrature, blocks, solvers).
"""
from .mesh import kuhn_mesh, kuhn_periodic_mesh, splitmix64_doubles
from .fields import (beltrami_velocity, beltrami_pressure, BeltramiParams, SolenoidalModes, abc_velocity,
                     abc_pressure)

__all__ = ["kuhn_mesh", "kuhn_periodic_mesh", "splitmix64_doubles", "beltrami_velocity", "beltrami_pressure",
           "BeltramiParams", "SolenoidalModes", "abc_velocity", "abc_pressure"]
