"""Seeded synthetic kernel models for the concrete-instance race check.

Shared by the CUDA path, the CPU oracle, the tests and the benchmark.  Nothing in
this package computes a race verdict: it only describes models.
"""
from .spec import (E, GLOBAL, SHARED, A, Access, Array, Expr, Loop, Model, R, Stmt, W, bid,
                   const, it, load, param, tid)
from .configs import (atomic_counter, atomic_histogram, batch_models, csr_row_lengths, grid_neighbor, grid_late_partner,
                      tiny_random_sync, warp_reduction, ge_spmm_csr, ge_spmm_uniform, neighbor_write_read,
                      permutation_scatter,
                      polyhedral_product,
                      random_affine, reduction_tree, request_stream, tiny_random, tiny_random_tables, transpose,
                      RANDOM_AFFINE_ROW_GLOBAL, RANDOM_AFFINE_ROW_SHARED)
from .rng import SplitMix64
