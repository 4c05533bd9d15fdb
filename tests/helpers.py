"""Shared test helpers (no method arithmetic)."""
import numpy as np


def field_scales(ref):
    """Per-field normalisation scales of the relative L1 error (one per field).

    rho: mean |rho|; momenta: sqrt(mean rho * mean E); E: mean |E|;
    face fields: rms |B|.  Fields whose mean is ~0 (momenta of a linear wave)
    are measured against these physical scales rather than their own L1 norm.
    """
    rho = float(np.mean(np.abs(ref[0])))
    e = float(np.mean(np.abs(ref[4])))
    m = float(np.sqrt(rho * e))
    b = float(np.sqrt(np.mean(ref[5] ** 2 + ref[6] ** 2 + ref[7] ** 2)))
    return np.array([rho, m, m, m, e, b, b, b])


def rel_l1(got, ref):
    """rel L1_f = sum|got - ref| / max(sum|ref|, N s_f) per field f."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    N = ref[0].size
    s = field_scales(ref)
    out = np.zeros(ref.shape[0])
    for f in range(ref.shape[0]):
        out[f] = np.sum(np.abs(got[f] - ref[f])) / max(np.sum(np.abs(ref[f])), N * s[f], 1e-300)
    return out
