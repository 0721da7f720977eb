"""FP64 CPU oracle of the MHD bunch update.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import anything from this package.  It shares no code with the CUDA path
(``paper_2508_09568_gb300``) and never imports it; both consume the seeded inputs of
``paper_2508_09568_gb300.workloads`` only through the tests that call them.

Parity status of each part: see the module docstrings of ``mhd`` and ``exact_riemann``
and the pins under ``tests/test_oracle_*.py``.
"""
