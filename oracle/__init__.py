"""FP64 CPU oracle for the multigrid Monge-Ampere reconstruction solve.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.
"""
