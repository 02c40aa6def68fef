"""CPU oracle for compressed-column queries.

TEST INFRASTRUCTURE: only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything here.  The product path
(the ``cq_*`` C-ABI library and its Python binding) never does.
"""
