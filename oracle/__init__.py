"""CPU oracle of the mining path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import anything from this package; the product path never does.
"""
