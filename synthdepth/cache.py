"""On-disk cache of generated sequences (the generator is deterministic per
workload seed; the cache only saves the host ray cast between runs)."""

from __future__ import annotations

import os

import numpy as np

from .configs import Sequence, make_sequence


def seq_cache_path(w, n, colour=False):
    d = os.environ.get("TSDF_SEQ_CACHE", "/tmp/tsdf_seq_cache")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"{w.name}_{w.seed}_{n}{'_rgb' if colour else ''}.npz")


def load_sequence(w, n, colour=False):
    """The first n frames of workload w's sequence (with colour images when
    asked), generated once and cached."""
    path = seq_cache_path(w, n, colour)
    if os.path.exists(path):
        z = np.load(path)
        return Sequence(workload=w, depth=z["depth"], poses=z["poses"], first_frame=0,
                        colour=z["colour"] if colour else None)
    seq = make_sequence(w, n_frames=n, colour=colour)
    try:
        extra = {"colour": seq.colour} if colour else {}
        np.savez(path + ".tmp.npz", depth=seq.depth, poses=seq.poses, **extra)
        os.replace(path + ".tmp.npz", path)
    except OSError:
        pass
    return seq
