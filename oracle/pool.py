"""Process-pool helper of the CPU baseline (TEST INFRASTRUCTURE ONLY, like the rest of this package): one
spawned process per host core decodes whole slots with the FP64 oracle chain, generating each slot (untimed)
just before decoding it, so that memory stays at one slot per process."""
from __future__ import annotations

import time


def decode_slots(task):
    """task = (workload preset name, slot indices, budget in seconds of decoding). Returns (slots decoded,
    seconds spent decoding)."""
    name, indices, budget_s = task
    from . import run_slot
    from paper_2210_09196_gb300 import synth
    done, spent = 0, 0.0
    for i in indices:
        s = synth.make_slot(synth.PRESETS[name], i)
        t0 = time.perf_counter()
        run_slot(s)
        spent += time.perf_counter() - t0
        done += 1
        if spent > budget_s:
            break
    return done, spent
