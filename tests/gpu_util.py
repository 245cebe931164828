"""Helpers shared by the GPU tests: move a synthetic cohort onto the device
(or keep it on the host) as a binding.SurvData, and build the matching
oracle inputs."""
import numpy as np
import scipy.sparse

from paper_2204_08183_gb300 import binding, synth


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def survdata(d, where="device"):
    """binding.SurvData for cohort dict ``d`` (dense or csc)."""
    put = dev if where == "device" else (lambda a: np.ascontiguousarray(a))
    t = put(d["time"])
    s = put(d["status"])
    if d["layout"] == "dense":
        X = d["X"]
        if where == "device":
            Xd = dev(np.ascontiguousarray(X.T))
        else:
            Xd = np.asfortranarray(X)
        return binding.SurvData(t, s, X=Xd)
    vals = d["values"]
    return binding.SurvData(t, s, col_ptr=put(d["col_ptr"]), row_idx=put(d["row_idx"]),
                            values=None if vals is None else put(vals), n=d["n"], p=d["p"])


def oracle_X(d):
    """X for the oracle: a dense ndarray or a scipy CSC matrix (float64)."""
    if d["layout"] == "dense":
        return d["X"]
    vals = d["values"] if d["values"] is not None else np.ones(d["row_idx"].shape[0])
    return scipy.sparse.csc_matrix((vals.astype(np.float64), d["row_idx"], d["col_ptr"]), shape=(d["n"], d["p"]))


def small_csc(n, p, seed, density=0.1, n_times=50, competing=0.0, binary=False, dtype=np.float32):
    """Small CSC cohort with arbitrary ties (and optional competing events)."""
    d = synth.cohort_small(n, p, seed, n_times=n_times, censor_frac=0.3, competing_frac=competing,
                           density=density)
    X = d["X"]
    if binary:
        X = (X != 0).astype(np.float64)
    col_ptr, row_idx, values = synth.csc_from_dense(X)
    return {"time": d["time"], "status": d["status"], "col_ptr": col_ptr, "row_idx": row_idx,
            "values": None if binary else values.astype(dtype), "n": n, "p": p, "layout": "csc",
            "beta": d["beta"], "X_dense": X}
