"""GB300-native mixed-basis (2D plane wave x B-spline) H/S apply and
generalized Lanczos-Krylov eigensolver (Ren, Hsue, Chang, arXiv:1406.4960).

The compute path is the CUDA library libmbgb300.so (C ABI in include/mb.h);
``paper_1406_4960_gb300.mb`` is its thin binding.  ``workloads`` holds the
seeded synthetic inputs."""

__all__ = ["mb", "workloads", "build"]
