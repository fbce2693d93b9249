"""FP64 CPU oracle for CTD.  Test infrastructure only: imported by tests/,
the smoke entry point and the benchmark's CPU-baseline leg, never by the
library."""
