"""GB300 (sm_103a) ACO library for large symmetric TSP instances -- Python binding.

Thin ctypes marshalling over the C ABI in ``include/aco.h`` (same entry-point names).  Every step
of the method runs in the library's CUDA kernels; PyTorch only provides device memory (tensor
``data_ptr()``) and streams.  Importing this package does not touch the GPU; the first call
loads ``lib/libaco_gb300.so`` and raises if it has not been built (``build.build()``).

The method is D. M. Chitty, "Applying ACO To Large Scale TSP Instances" (UKCI 2017):
Section 2 (Eq. 1-5), Section 3 (l_best pheromone, weights C_gbest / C_lbest) and Section 3.1
(PartialACO, Algorithm 1).
"""
from __future__ import annotations

import ctypes
import os

from ._ffi import (ACO_MODE_DENSE, ACO_MODE_LBEST_PARTIAL, AcoError, Params, Stats, lib, library_path)
from .colony import Colony

__all__ = [
    "ACO_MODE_DENSE", "ACO_MODE_LBEST_PARTIAL", "AcoError", "Params", "Stats", "Colony", "lib", "library_path",
    "aco_create_instance", "aco_build_candidates", "aco_construct_tours", "aco_update_pheromone",
    "aco_tour_lengths", "aco_get_state", "aco_set_state", "aco_get_stats", "aco_step_probs",
    "aco_destroy_instance", "aco_build_candidates_noalloc", "aco_batch_create", "aco_batch_build_candidates",
    "aco_batch_run", "aco_batch_get_state", "aco_batch_get_best", "aco_batch_schedule", "aco_batch_destroy",
    "Batch", "aco_batch_instance", "ACO_MLP_WEIGHTS", "aco_mlp_create", "aco_mlp_get_weights", "aco_mlp_forward",
    "aco_mlp_backward", "aco_mlp_adam", "aco_mlp_train", "aco_mlp_destroy", "aco_edge_features", "aco_tour_labels",
    "aco_set_edge_scores", "EdgeScorer", "aco_set_max_mod_frac", "aco_set_p_partial", "linear_f_schedule",
    "aco_set_local_search",
    "aco_set_async_share", "aco_probe_bandwidth", "aco_set_ant_range", "aco_export_commits", "aco_import_commits",
    "ShardedColony", "exchange_records", "aco_batch_set_schedule", "aco_batch_set_wait_limit", "ACO_BATCH_SCHEDULES",
]

from .batch import Batch  # noqa: E402
from ._ffi import (aco_batch_build_candidates, aco_batch_create, aco_batch_destroy, aco_batch_get_best,  # noqa: E402
                   aco_batch_get_state, aco_batch_run, aco_batch_schedule)
from ._ffi import aco_export_commits, aco_import_commits, aco_probe_bandwidth, aco_set_ant_range  # noqa: E402
from ._ffi import ACO_BATCH_SCHEDULES, aco_batch_set_schedule, aco_batch_set_wait_limit  # noqa: E402
from .sharded import ShardedColony, exchange_records  # noqa: E402
from ._ffi import (aco_build_candidates, aco_build_candidates_noalloc, aco_construct_tours, aco_create_instance, aco_destroy_instance,  # noqa: E402
                   aco_get_state, aco_get_stats, aco_set_state, aco_step_probs, aco_tour_lengths,
                   aco_update_pheromone)
from ._ffi import (ACO_MLP_WEIGHTS, aco_batch_instance, aco_edge_features, aco_mlp_adam,  # noqa: E402
                   aco_mlp_backward, aco_mlp_create, aco_mlp_destroy, aco_mlp_forward, aco_mlp_get_weights,
                   aco_mlp_train, aco_set_edge_scores, aco_tour_labels)
from .learned import EdgeScorer  # noqa: E402
from ._ffi import aco_set_async_share, aco_set_local_search, aco_set_max_mod_frac, aco_set_p_partial  # noqa: E402
from .colony import linear_f_schedule  # noqa: E402
