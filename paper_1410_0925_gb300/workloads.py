"""Call schedules of the measured workloads that are more than one library
call per frame (shared by the benchmark and the profiling drivers)."""

# near plane of the raycast search range in the raycast workloads (metres)
Z_NEAR = 0.2
# swapping workload: blocks moved per call at most, and the view margin (pixels)
SWAP_CAPACITY = 4096
SWAP_MARGIN_PX = 16.0


def swap_step_ops(scene, depth_dev, intr, poses):
    """One frame schedule of the swapping workload: bring back what the view
    sees, fuse, move out what it does not (Section 5)."""
    for i in range(depth_dev.shape[0]):
        scene.swap_in(intr, poses[i], SWAP_MARGIN_PX)
        scene.integrate(depth_dev[i], intr, poses[i])
        scene.swap_out(intr, poses[i], SWAP_MARGIN_PX)
