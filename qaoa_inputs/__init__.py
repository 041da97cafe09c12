"""Seeded synthetic problem instances shared by the CPU oracle and the CUDA path.

This package draws random numbers only: graphs, couplings, angles and batch
recipes. It holds none of the QAOA arithmetic (no cost functions, no states,
no mixers), so that the oracle and the GPU implementation stay independent.
"""

from .generators import (  # noqa: F401
    BASE_SEED,
    erdos_renyi,
    ramp_angles,
    random_regular3,
    sk_couplings,
    uniform_angles,
    uniform_angles_ma,
    uneven_batch_recipe,
    WORKLOADS,
    workload_instance,
)
