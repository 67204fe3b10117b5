"""Seeded synthetic inputs: check matrices and sampled errors/syndromes.

Nothing here performs decoding; both the CUDA path and the CPU oracle take
these inputs as plain arrays.
"""
from .codes import (SparseH, rotated_surface, unrotated_surface, spacetime,
                    spacetime_priors, bivariate_bicycle, bb_code, gf2_rank,
                    logical_operators)
from .sampler import sample, pack, unpack, words

__all__ = ["SparseH", "rotated_surface", "unrotated_surface", "spacetime",
           "spacetime_priors", "bivariate_bicycle", "bb_code", "gf2_rank",
           "logical_operators", "sample", "pack", "unpack", "words"]
