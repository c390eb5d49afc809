"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

Holds workload records and the Zel'dovich initial-condition generator only;
none of the force method's arithmetic lives here."""
from .workloads import C1, C2, C2_MID, C2_SMALL, C3, C5, WORKLOADS, Level, Workload  # noqa: F401
