"""FP64 CPU oracles of the FCFS block transform -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_1010_5562_gb300``) and never imports it.

* ``fcfs_oracle`` (O1): the direct vertex sum with full tail integrals, the
  gradient formulas and the pupil loss -- the reference every GPU result is
  compared with.
* ``edge_form`` (O2): Prop. CFT over clockwise rings.
* ``sparse_fft`` (O4): Steps 1-4 of FCFS with numpy's FFT.
* ``brute`` (O3): unit-cell rasterisation plus quadrature, tiny periods only.
* ``cosine``: the continuous cosine series (direct vertex sum with full tails).
* ``haar``: the pruned continuous Haar transform (per-polygon recursion with Alg. 1).
"""
from . import fcfs_oracle, edge_form, sparse_fft, brute, cosine, haar
from .fcfs_oracle import (block, block_entries, tail_integral, area_exact, pupil_mask,
                          pupil_loss, vertex_gradient, edge_gradient, relative_error, freqs)
from .cosine import cosine_block, cosine_entries
from .haar import pcht
