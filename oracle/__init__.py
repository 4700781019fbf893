"""FP64 CPU oracle of Progressively Projected Newton (test infrastructure only).

The product library never imports this package.  Only ``tests/``, the smoke
check in ``__graft_entry__`` and ``bench.py``'s CPU-baseline leg use it.
"""
