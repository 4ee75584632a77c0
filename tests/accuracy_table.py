#!/usr/bin/env python3
"""Final-DVF error of the GPU registration against the FP64 oracle, per
configuration and image storage type (FP32 / FP16 / BF16; the oracle always
runs on the FP32 images).  Test infrastructure, run by hand on a machine with a GB300:

    python tests/accuracy_table.py [--full] > accuracy.json

(--full runs the 512 x 512 x 160 case for its whole 100/50/25 iterations:
about 7 minutes of the oracle on 16 host cores.)

Prints one JSON object: per case the RMS difference over the whole volume
and over the body, in voxels, beside the RMS of the ground-truth DVF.
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    """DVF error of the GPU registration against the FP64 oracle, per config
    and image storage type (the oracle always runs on the FP32 images)."""
    import numpy as np
    import torch

    import oracle
    import paper_1301_0970_gb300 as cg
    import phantom

    dev = torch.device("cuda", 0)
    full = "--full" in sys.argv            # the pelvic case at its full 100/50/25 iterations
    runs = [("phantom64", None, 1, [100]), ("headneck256", None, 3, [100, 50, 25]),
            ("pelvis512", None, 3, [100, 50, 25] if full else [10, 5, 2])]
    out = {}
    with cg.Context(0) as ctx:
        for name, shape, levels, iters in runs:
            c = phantom.make_case(name, shape=shape)
            t0 = time.perf_counter()
            ref, _ = oracle.register(c.static, c.moving, c.static_masks, c.moving_masks, levels=levels,
                                     iters=iters, lam=c.lam, sign=c.signs, stop_mode=oracle.STOP_FIXED)
            t_oracle = time.perf_counter() - t0
            row = {"iters": iters, "oracle_seconds": round(t_oracle, 2)}
            body = c.body.astype(bool)
            for label, code in (("f32", cg.CGDIR_F32), ("f16", cg.CGDIR_F16), ("bf16", cg.CGDIR_BF16)):
                dvf, _ = ctx.register(torch.from_numpy(c.static).to(dev), torch.from_numpy(c.moving).to(dev),
                                      [torch.from_numpy(m).to(dev) for m in c.static_masks],
                                      [torch.from_numpy(m).to(dev) for m in c.moving_masks],
                                      levels=levels, iters=iters, lam=c.lam, sign=c.signs,
                                      stop_mode=cg.CGDIR_STOP_FIXED, storage_dtype=code)
                d2 = ((dvf.cpu().numpy().astype(np.float64) - ref) ** 2).sum(axis=0)
                row[label] = float(np.sqrt(d2.mean()))
                row[label + "_body"] = float(np.sqrt(d2[body].mean()))
            gt = np.sqrt((c.u_gt.astype(np.float64) ** 2).sum(axis=0).mean())
            row["rms_u_gt"] = float(gt)
            row["body_fraction"] = float(body.mean())
            out[f"{name} {'x'.join(map(str, c.shape[::-1]))}"] = row
    print(json.dumps({"dvf_rms_error_vs_fp64_oracle_voxels": out}), flush=True)
    return 0



if __name__ == "__main__":
    sys.exit(main())
