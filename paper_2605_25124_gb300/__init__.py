"""GB300-native (sm_103a) Gini multidimensional scaling.

The compute path is libginimds.so (hand-written CUDA kernels behind a C ABI,
include/gini_mds.h); this package is its thin Python binding.  `workloads`
holds the seeded synthetic input generators.
"""
from .api import (Dissimilarity, GiniStress, Workspace, default_step, deterministic, fit_host,
                  gini_alternating_nu, gini_classical_mds, gini_delta_sums, gini_dist,
                  gini_distance_correlations, gini_fit_batched, gini_mds_fit,
                  gini_neighbour_scores, gini_nu_search, gini_pack, gini_rank, gini_silhouette,
                  gini_stress, gini_stress_grad, is_deterministic, tile_size, tiled_elems,
                  workspace, workspace_size)

__all__ = ["Dissimilarity", "GiniStress", "Workspace", "default_step", "deterministic",
           "fit_host", "gini_alternating_nu", "gini_classical_mds", "gini_delta_sums",
           "gini_dist", "gini_distance_correlations", "gini_fit_batched", "gini_mds_fit",
           "gini_neighbour_scores", "gini_nu_search", "gini_pack", "gini_rank",
           "gini_silhouette", "gini_stress", "gini_stress_grad", "is_deterministic",
           "tile_size", "tiled_elems", "workspace", "workspace_size"]
