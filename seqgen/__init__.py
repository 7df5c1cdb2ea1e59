"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

Holds random draws and scoring tables only (no alignment arithmetic).
"""
from .matrices import (blosum62, dna_matrix, aa_background, PROTEIN_LETTERS,
                       STANDARD_AA, DNA_LETTERS)
from .synth import (WORKLOADS, Workload, generate, scoring, random_sequences,
                    reference_sample, training_pairs, split_sequences, pack_sequences)
