"""Plain FP64 CPU oracle of (triad-)ATRG — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import anything from this package.  The product
path (``paper_2507_21909_b300``) never imports it and shares no code with it.
"""
