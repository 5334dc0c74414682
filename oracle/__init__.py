"""FP64 CPU oracle for the AFiD pressure-correction hot path.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
execute anything in this package. The product path (the CUDA library and its
Python binding) never touches it and shares no code with it.

This is a plain, slow, obviously-correct restatement of what the paper's solver
computes (AFiD, arXiv 1705.01423), written in PyTorch CPU float64 ops:

  grid.py      stretched staggered grid and its metric (Sec. 2.1, Fig. 1)
  operators.py divergence, gradient, Laplacian, wall-normal second differences,
               conservative advection, horizontal diffusion, CFL (Sec. 2.1,
               Listing 1)
  poisson.py   the Fourier-Thomas Poisson solve (Sec. 2.2, the twelve-step
               algorithm with its transposes dropped)
  timestep.py  pressure correction, low-storage RK3 + Crank-Nicolson substep,
               Nusselt number (Sec. 2.1, Sec. 2.2 last paragraph)
  adjoint.py   reverse-mode derivatives of the above by automatic
               differentiation of the very same forward code
  stats.py     wall-normal statistics: horizontal means per plane, Nusselt
               numbers, wall shear stress, friction Reynolds number (Sec. 3.2,
               Sec. 5)
  sampled.py   the Poisson solve at a few wavenumber pairs (large grids)
  multires.py  temperature on a refined grid with a refined time step:
               fine grid, trilinear prolongation of the velocity, restriction
               of the temperature, the coupled step (Sec. 6)

Coordinates follow the workloads, not the paper: x and y are the periodic,
uniform directions and z is the bounded, stretched wall-normal direction (the
paper calls the wall-normal direction x, Sec. 2.1). Arrays are C-ordered
[z][y][x].

Every function here is pinned by tests that do not reuse its own formulas
(closed-form discrete eigenpairs, dense brute-force solves on 8^3 grids, exact
steady states, conservation identities, Runge-Kutta order conditions and
finite differences).
"""
from .grid import Grid
from . import operators, poisson, timestep, adjoint, multires

__all__ = ["Grid", "operators", "poisson", "timestep", "adjoint", "multires"]
