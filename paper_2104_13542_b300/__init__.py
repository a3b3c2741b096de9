"""B300-native (sm_103a) STORM joint-space sampling-based MPC control step.

The control step of Bhardwaj et al. (arXiv 2104.13542, Algorithm 1) runs in the
CUDA library ``libstorm_b300.so`` behind the C ABI of ``include/storm.h``;
``binding`` is its ctypes marshalling layer and ``workloads`` draws seeded
synthetic inputs shaped like the paper's.
"""
from .binding import (BatchController, Controller, StormError, SurrogateMLP, build,  # noqa: F401
                      lib, status_string, storm_cost)

__all__ = ["BatchController", "Controller", "StormError", "SurrogateMLP", "build", "lib",
           "status_string", "storm_cost"]
