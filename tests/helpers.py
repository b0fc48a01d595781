"""Shared helpers of the test suite (no arithmetic of the method here)."""
import numpy as np


def force_error(e, e64):
    """Floored relative field error per target: |E - E64| / max(|E64|, rms|E64|)
    (the rms floor avoids dividing by nearly cancelled fields).  Returns the
    per-target errors."""
    e = np.asarray(e, np.float64).reshape(-1, 3)
    e64 = np.asarray(e64, np.float64).reshape(-1, 3)
    nrm = np.linalg.norm(e64, axis=1)
    rms = np.sqrt(np.mean(nrm ** 2))
    return np.linalg.norm(e - e64, axis=1) / np.maximum(nrm, rms)


def summary(err):
    return {"median": float(np.median(err)), "p99": float(np.percentile(err, 99)),
            "max": float(np.max(err))}


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
