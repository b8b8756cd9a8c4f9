"""FP64 CPU oracle of the colloidal Shan-Chen lattice-Boltzmann step.

Test infrastructure only: the tests, the package smoke check and the CPU
baseline leg of the benchmark load it; the product path never does.
"""
from .oracle import Oracle, build_oracle, lattice, feq, pair_force, integrate_one, OrcParams, set_threads

__all__ = ["Oracle", "build_oracle", "lattice", "feq", "pair_force", "integrate_one", "OrcParams", "set_threads"]
