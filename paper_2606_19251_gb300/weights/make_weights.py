"""Train the GCIN on the synthetic training batch and write gcin_c3.npy.

Training batch: 64 Delaunay finite-volume meshes of 2k-20k nodes cycling
uniform / 10:1 graded / graded + anisotropic band (aspect <= 100) point
sets (workloads.c3_batch, seed 0); validation: 8 more meshes of the same
distribution (seed 1).  Algorithm 1 with the multi-V-cycle loss (N_vc = 3 by default), mini-batch 5, Adam lr
1e-3, clipping 1.0, ReduceLROnPlateau, best-validation parameters kept
(Table train_hyper).  Every forward/backward runs on the GPU through
libamggnn.so.

    python -m paper_2606_19251_gb300.weights.make_weights [--epochs 150]

gcin_wide.npy (the parameters used for the anisotropic band and airfoil
workloads) comes from the same run with the distribution widened by 16 band
meshes of aspect ratio up to 1000 and 16 small airfoil meshes:

    python -m paper_2606_19251_gb300.weights.make_weights --extra-band1000 16 --extra-airfoil 16 \
        --out paper_2606_19251_gb300/weights/gcin_wide.npy

gcin_c3_h32.npy is the halved GCIN width of App. B.3 (37,189 parameters)
trained on the same C3 batch:

    python -m paper_2606_19251_gb300.weights.make_weights --hidden 32 \
        --out paper_2606_19251_gb300/weights/gcin_c3_h32.npy

gcin_struct.npy / gcin_struct_h32.npy are trained on Cartesian grids with
immersed bodies (workloads.structured_batch: 64 training and 8 validation
grids, 2D and 3D), the setting App. B.3 halves the width for:

    python -m paper_2606_19251_gb300.weights.make_weights --dataset structured [--hidden 32] \
        --out paper_2606_19251_gb300/weights/gcin_struct[_h32].npy
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--batch", type=int, default=5)
    ap.add_argument("--meshes", type=int, default=64)
    ap.add_argument("--nvc", type=int, default=3, help="V-cycles per loss (Sec. 3.3 multi-V-cycle loss)")
    ap.add_argument("--val-cycles", type=int, default=10)
    ap.add_argument("--extra-band1000", type=int, default=0,
                    help="add this many graded + band meshes with aspect ratios up to 1000")
    ap.add_argument("--extra-airfoil", type=int, default=0,
                    help="add this many small airfoil meshes (wall layers from 1e-5 chords)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"],
                    help="arithmetic of the forward node linears during training")
    ap.add_argument("--hidden", type=int, default=64, choices=[64, 32], help="GCIN width (App. A.1: 64; App. B.3: 32)")
    ap.add_argument("--dataset", default="c3", choices=["c3", "structured"],
                    help="C3 unstructured meshes or Cartesian grids with immersed bodies")
    ap.add_argument("--out", default=os.path.join(HERE, "gcin_c3.npy"))
    args = ap.parse_args()
    import workloads as W
    from paper_2606_19251_gb300 import _build
    from paper_2606_19251_gb300.train import train
    _build.build()
    t0 = time.time()
    if args.dataset == "structured":
        mats = W.structured_batch(args.meshes, seed=0)
        val = W.structured_batch(8, seed=1)
    else:
        mats = W.c3_batch(args.meshes, seed=0)
        val = W.c3_batch(8, seed=1)
    # optional widening of the training distribution (not part of the C3 batch)
    for k in range(args.extra_band1000):
        n = int(2000 + 18000 * W.uniform01(7000 + k, 1)[0])
        mats.append(W.fv_mesh("band", n, 7000 + k, max_aspect=1000.0)[0])
    for k in range(args.extra_airfoil):
        mats.append(W.c5_problem(8000 + k, n_rhs=1, n_surface=160, n_far=4000 + 500 * k)[0])
    print(f"meshes ready in {time.time() - t0:.1f}s: n = {[m.n_rows for m in mats[:8]]}...", flush=True)
    theta0 = W.gcin_init_params(0, hidden=args.hidden)
    from paper_2606_19251_gb300 import api as P
    prec = P.AMG_GNN_BF16 if args.precision == "bf16" else P.AMG_GNN_FP32
    best, rows = train(mats, val, theta0, epochs=args.epochs, batch=args.batch, n_vc=args.nvc,
                       val_cycles=args.val_cycles, log=lambda r: print(json.dumps(r), flush=True), precision=prec)
    np.save(args.out, np.asarray(best, dtype=np.float32))
    # the training log is run output, not a product file: it goes beside the
    # run's other output (LOG_DIR, default the working directory)
    log_dir = os.environ.get("LOG_DIR", os.getcwd())
    with open(os.path.join(log_dir, os.path.basename(os.path.splitext(args.out)[0]) + "_log.json"), "w") as f:
        json.dump({"epochs": args.epochs, "batch": args.batch, "meshes": args.meshes, "n_vc": args.nvc,
                   "extra_band1000": args.extra_band1000, "extra_airfoil": args.extra_airfoil,
                   "precision": args.precision, "hidden": args.hidden, "dataset": args.dataset,
                   "val_cycles": args.val_cycles, "rows": rows,
                   "seconds": time.time() - t0}, f, indent=1)
    print("wrote", args.out, flush=True)


if __name__ == "__main__":
    main()
