"""Several independent searches of one instance, keeping the best (Sec. 4.1).

Sec. 4.1 builds alternative initial orders by shuffling the activities of each
level.  Each start is the instance with its own shuffle keys
(`instances.level_keys(inst, seed + k)`); rcpsp_multistart runs all starts
as independent searches in one launch and keeps the best final makespan,
ties to the lowest start index.  This module only draws the keys (inputs)
and marshals the call.
"""
from __future__ import annotations


def multistart(solver, inst, starts: int, seed: int = 0, iterations: int = 1000, delta: int = 0,
               tabu_len: int = 0, mode: int = 0, stream=None, first_unshuffled: bool = True) -> dict:
    """Runs `starts` searches of `inst`; returns the best result plus every start's makespan.

    With `first_unshuffled`, start 0 uses the unshuffled level order (the
    default initial list) and starts 1.. use shuffle keys seed+1, seed+2, ...
    """
    from .instances import level_keys
    keys = [None if (first_unshuffled and k == 0) else level_keys(inst, seed + k) for k in range(starts)]
    out = solver.multistart(inst, keys, iterations=iterations, delta=delta, tabu_len=tabu_len, mode=mode,
                            stream=stream)
    out["keys"] = keys
    return out
