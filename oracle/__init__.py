"""FP64 CPU oracle of the coupled phase-field lattice Boltzmann time step.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. The product path (the
CUDA library and its Python binding) never imports, links or executes
anything here, and nothing here imports the product path.

The oracle restates, in plain numpy at float64, the equations of
"Comparative study and critical assessment of phase-field lattice Boltzmann
models for laminar and turbulent two-phase flow simulations" (arXiv
2511.11360): Sec. II B (the shared BGK lattice Boltzmann equations), Sec. II C
(Fakhari2017, Liang2018, Chai2018, Hu2019), Sec. II D (Liang2014), and the isotropic
central stencils of Sec. III. Every function cites the passage it follows.
Readings of passages the paper leaves silent or ambiguous are marked
``Reading R<n>``; the list is kept in the repository's design notes.

Parity pins (tests/test_oracle_*.py) fix every part of it against closed
forms, invariants and the paper's printed numbers; none is "unpinned".
"""

from .pflb_oracle import *  # noqa: F401,F403
