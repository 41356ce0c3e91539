"""Plain, slow FP64 CPU oracle of the solid Newton step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` use it.  It shares no code
with the CUDA path; the seeded input generators in ``fixtures`` are the only
common ground.
"""
from . import solid  # noqa: F401
