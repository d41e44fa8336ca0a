"""CPU oracle for the ranking / order-statistic / sorting circuits under RNS-CKKS.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product library never does.
"""
