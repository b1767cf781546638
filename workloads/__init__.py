"""Seeded synthetic inputs (geometries, boundary data, workloads) shared by the
tests, the benchmark and the CPU oracle.  No IBDL arithmetic lives here."""
from . import configs, data, geometry  # noqa: F401
