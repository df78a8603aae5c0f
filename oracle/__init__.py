"""Sequential CPU oracle for the round-based independent-set mesh adaptation.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the product library never does.
"""
