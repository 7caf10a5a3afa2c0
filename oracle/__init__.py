"""FP64 CPU oracle of the exponential-integrator hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import anything under ``oracle/``.
The product library never imports, links or calls it, and the oracle shares no code
with the CUDA path (it takes plain numpy arrays as inputs).

Modules:
  adr_oracle  -- grid operators, matrix functions and the time integrators.
"""
