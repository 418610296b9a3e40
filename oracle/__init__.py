"""CPU oracle for the selection library (test infrastructure only).

Plain, slow, obviously correct restatements of what the GPU path computes, written
from G. Beliakov, "Parallel calculation of the median and order statistics on GPUs
with application to robust regression" (arXiv:1104.2732).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package.  The GPU library never imports, links or runs
anything from here, and nothing here imports the GPU library: the two share no code.
Arithmetic is float64 unless a function says otherwise.

Modules
-------
select      exact order statistics, counts, the pinball cost, Kelley's cutting plane
regression  LMS / LTS objectives of robust regression
knn         k-nearest-neighbour regression and classification through d_(k)
bracket     sketch features and the bracket-proposal MLP (float64 forward/backward)
philox      the Philox4x32-10 counter-based generator (for the training-data generator)
"""
from . import select, regression, knn, bracket, philox  # noqa: F401
