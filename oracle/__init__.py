"""FP64 CPU oracle of the per-day DODE / SPGD path -- test infrastructure only.

Imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py``; never by the product package.
"""
