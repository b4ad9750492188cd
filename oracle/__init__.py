"""CPU oracle for the AP IMEX-RK D2V6 scheme.  Test infrastructure only:
imported by tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py``; never by the product library or its binding."""
