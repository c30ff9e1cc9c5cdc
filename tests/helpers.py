"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


def gpu_trace(trace_tensor, s, n_face):
    return trace_tensor[s, :, :n_face].double().cpu().numpy()
