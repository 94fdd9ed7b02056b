"""Seeded synthetic inputs for the FC-DOM RTE solver: grids, media, beams and
detectors.  This module holds no arithmetic of the method itself; both the
oracle (tests) and the CUDA library's callers (tests, bench) draw their inputs
from here, so that each side computes everything else on its own."""
from .workloads import (Beam, Detector, Grid, Optics, Workload, face_point,
                        perimeter_detectors, workload_small, workload_tomo256,
                        workload_precision512, workload_mss256, workload_batched,
                        workload_custom, workload_inverse, add_relative_noise)

__all__ = ["Beam", "Detector", "Grid", "Optics", "Workload", "face_point",
           "perimeter_detectors", "workload_small", "workload_tomo256",
           "workload_precision512", "workload_mss256", "workload_batched",
           "workload_custom", "workload_inverse", "add_relative_noise"]
