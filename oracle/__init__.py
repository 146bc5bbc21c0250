"""FP64 CPU oracle of the Cool-chic overfitting iteration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package.  It shares no code with the CUDA library in
``paper_2403_11651_gb300`` and never imports it.
"""
