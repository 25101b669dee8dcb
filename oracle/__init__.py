"""CPU oracle for the Pauli-sum product -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The GPU library never imports, links or calls it.
"""
