"""Training and evaluation of the learned NCC-weight network (pam_learn_*).

The network is trained on frames the method itself turns into examples:
synthetic channel data of the 128-element workload go through
``pam_learn_example``, which returns the network input (band energies of the
full-aperture AS map, Eq. 3) and the target (the exact rho_TAX of Eq. 4 and
Eq. 10). Forward, backward and Adam run in libpam's kernels
(``pam_learn_train_step``).

Training frames: the receive model is linear in the sources, so frames are
made as sums of 1-6 single-source responses drawn from a seeded bank
(``synth.source_response``), each with a seeded gain, plus white channel noise
at 20 dB SNR. Superposition and noise are input synthesis; they are done on
the GPU with torch so that 20k frames take seconds. Held-out frames come from
``synth.make_frame`` (independent sources and seeds).

  python -m paper_2412_02413_gb300.learn [--frames 20000] [--epochs 3] [--out PATH]
      [--checkpoint PATH --checkpoint-every N] [--resume PATH]

Checkpoint and resume: the training state (parameters, Adam moments, step)
is saved every N steps; --resume restores it, rebuilds the same seeded
examples and batch order, and continues from the saved step. The kernels
reduce in a fixed order, so a resumed run reproduces the uninterrupted one.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CHECKPOINT = os.path.join(HERE, "weights", "ncc_cnn_astax_128el_128x512.npz")
BANK_SEED = 1_000_000        # sources of the training bank
HELD_OUT_FIRST = 500_000     # frame indices of the held-out synth.make_frame frames


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights and zero biases, flat in the library's order
    (per layer w[out][in][3][3] then b[out])."""
    rng = np.random.default_rng(seed)
    chans = (5, 32, 32, 32, 32, 1)
    parts = []
    for cin, cout in zip(chans[:-1], chans[1:]):
        parts.append((rng.standard_normal((cout, cin, 3, 3)) * math.sqrt(2.0 / (9 * cin))).ravel())
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)


def _response(args):
    w, src, seed = args
    return synth.source_response(w, src, seed)


def make_bank(w, n: int, seed: int = BANK_SEED, workers: int = 0) -> np.ndarray:
    """[n][n_elem][nt] float32 single-source responses (spawned worker pool)."""
    srcs = synth.bank_sources(w, n, seed)
    jobs = [(w, s, seed + 7 + i) for i, s in enumerate(srcs)]
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    if workers == 1:
        return np.stack([_response(j) for j in jobs])
    with mp.get_context("spawn").Pool(workers) as pool:
        return np.stack(pool.map(_response, jobs, chunksize=8))


def mix_frames(bank, n: int, gen, max_sources: int = 6, snr_db: float = 20.0):
    """n frames [n][n_elem][nt] on the bank's device: sums of 1..max_sources
    bank responses with gains in [0.6, 1.4], plus white noise at snr_db
    relative to each frame's mean channel power."""
    import torch
    dev = bank.device
    K = bank.shape[0]
    count = torch.randint(1, max_sources + 1, (n,), generator=gen, device=dev)
    idx = torch.randint(0, K, (n, max_sources), generator=gen, device=dev)
    gain = 0.6 + 0.8 * torch.rand((n, max_sources), generator=gen, device=dev)
    rf = torch.zeros((n,) + tuple(bank.shape[1:]), dtype=torch.float32, device=dev)
    for j in range(max_sources):
        g = gain[:, j] * (count > j).float()
        rf += g[:, None, None] * bank.index_select(0, idx[:, j])
    p = rf.pow(2).mean(dim=(1, 2))
    sigma = torch.sqrt(p / 10.0 ** (snr_db / 10.0))
    rf += torch.randn(rf.shape, generator=gen, device=dev) * sigma[:, None, None]
    return rf


def save_checkpoint(path: str, params: np.ndarray, meta: dict):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=np.asarray(params, np.float32), meta=np.array(json.dumps(meta)))


def load_checkpoint(path: str = CHECKPOINT):
    d = np.load(path)
    return d["params"], json.loads(str(d["meta"]))


def save_training_state(path: str, learned, step: int, meta: dict):
    """Parameters, Adam moments and the step reached (written atomically)."""
    state, adam_steps = learned.get_state()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp.npz"
    np.savez(tmp, state=state, adam_steps=np.int64(adam_steps), step=np.int64(step), meta=np.array(json.dumps(meta)))
    os.replace(tmp, path)


def load_training_state(path: str):
    d = np.load(path)
    return d["state"], int(d["adam_steps"]), int(d["step"]), json.loads(str(d["meta"]))


def batch_schedule(n_batches: int, epochs: int, seed: int):
    """Batch index of every step: a seeded permutation per epoch."""
    import torch
    gen = torch.Generator().manual_seed(seed)
    return [b for _ in range(epochs) for b in torch.randperm(n_batches, generator=gen).tolist()]


def lr_at(step: int, steps: int, lr: float, lr_min: float) -> float:
    """Cosine decay from lr to lr_min over the run."""
    return lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * step / steps))


def held_out_frames(w, n: int, first: int = HELD_OUT_FIRST, workers: int = 0) -> np.ndarray:
    jobs = [(w, first + i) for i in range(n)]
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return np.stack(pool.map(_frame, jobs))


def _frame(args):
    w, f = args
    return synth.make_frame(w, f)[0]


STRICT_REL_L2 = 1e-2   # accuracy bar of a chosen form: rel L2 of the normalised image, peak pixel exact


def accuracy_rows(img_l, img_t, img_as, gate_err, gate_pass, w):
    """Per-frame accuracy of learned images img_l against exact AS-TAX img_t
    (device [F][nz][nx]): relative L2 of the max-normalised images over every
    pixel, brightest-pixel agreement, whether the frame meets the strict bar
    (rel L2 <= 1e-2 with the exact peak), and the Eq. 12 ISNR / A_0.5 of the
    learned, exact and plain AS images from pam_image_metrics (GPU)."""
    import torch
    from . import pam
    x0 = -(w.nx - 1) / 2 * w.pitch
    m = {k: pam.image_metrics(v, x0, w.pitch, w.z0, w.dz) for k, v in
         (("learned", img_l), ("tax", img_t), ("as", img_as))}
    nl = img_l / img_l.amax(dim=(1, 2), keepdim=True)
    nt = img_t / img_t.amax(dim=(1, 2), keepdim=True)
    rel = (torch.linalg.vector_norm(nl - nt, dim=(1, 2)) / torch.linalg.vector_norm(nt, dim=(1, 2))).cpu().numpy()
    pl = img_l.flatten(1).argmax(1).cpu().numpy()
    pt = img_t.flatten(1).argmax(1).cpu().numpy()
    ge, gp = gate_err.cpu().numpy(), gate_pass.cpu().numpy()
    rows = []
    for f in range(img_l.shape[0]):
        rows.append({
            "gate_err": float(ge[f]), "gate_pass": int(gp[f]), "rel_l2": float(rel[f]),
            "peak_match": bool(pl[f] == pt[f]),
            "meets_bar": bool(rel[f] <= STRICT_REL_L2 and pl[f] == pt[f]),
            "isnr_learned": m["learned"][f]["isnr_db"], "isnr_tax": m["tax"][f]["isnr_db"],
            "isnr_as": m["as"][f]["isnr_db"], "esa_learned": 1e6 * m["learned"][f]["esa_m2"],
            "esa_tax": 1e6 * m["tax"][f]["esa_m2"], "esa_as": 1e6 * m["as"][f]["esa_m2"],
        })
    return rows


def evaluate(learned, plan, rf_t, w, gate_tol: float):
    """Learned vs plain AS-TAX on frames rf_t (accuracy_rows per frame)."""
    import torch
    learned.configure(gate_tol=gate_tol, tensor_cores=True)
    out = learned.as_tax(rf_t)
    ref = plan.as_tax(rf_t, rho_n=True, image_as=True)
    torch.cuda.synchronize()
    return accuracy_rows(out["image"], ref["image"], ref["image_as"], out["gate_err"], out["gate_pass"], w)


def summarize(rows):
    """Means over the frames; the accepted_* entries cover the frames that
    passed the gate, the only ones whose learned image is returned."""
    a = lambda k, rs=rows: float(np.mean([r[k] for r in rs])) if rs else float("nan")
    acc = [r for r in rows if r["gate_pass"]]
    return {"frames": len(rows), "gate_pass_rate": a("gate_pass"), "gate_err_median": float(np.median(
        [r["gate_err"] for r in rows])), "rel_l2_mean": a("rel_l2"), "peak_match_rate": a("peak_match"),
        "meets_bar_rate": a("meets_bar"),
        "accepted_rel_l2_max": float(max([r["rel_l2"] for r in acc], default=float("nan"))),
        "accepted_meet_bar": bool(all(r["meets_bar"] for r in acc)),
        "isnr_learned_db": a("isnr_learned"), "isnr_tax_db": a("isnr_tax"), "isnr_as_db": a("isnr_as"),
        "esa_learned_mm2": a("esa_learned"), "esa_tax_mm2": a("esa_tax"), "esa_as_mm2": a("esa_as")}


def train(args):
    import torch
    from . import pam
    torch.cuda.set_device(0)
    w = synth.workload(2)
    t0 = time.time()
    bank_np = make_bank(w, args.bank, workers=args.workers)
    bank = torch.from_numpy(bank_np).cuda()
    del bank_np
    t_bank = time.time() - t0
    G = args.gen_batch
    L = pam.Learned.from_workload(w, max_frames=G)
    L.set_params(init_params(args.seed))
    N = args.frames
    feats = L.empty_features(N)
    target = torch.empty((N, w.nz, w.n_elem), dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(args.seed + 17)
    t1 = time.time()
    for s in range(0, N, G):
        n = min(G, N - s)
        rf = mix_frames(bank, n, gen)
        L.example(rf, features=feats[s:s + n], target=target[s:s + n])
    L.sync()
    t_data = time.time() - t1
    del bank
    B = args.batch
    nb = N // B
    steps = args.epochs * nb
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    schedule = batch_schedule(nb, args.epochs, args.seed + 29)
    log = []
    start = 0
    if args.resume:
        state, adam_steps, start, _ = load_training_state(args.resume)
        L.set_state(state, adam_steps)
    t2 = time.time()
    for step in range(start, steps):
        bi = schedule[step]
        L.train_step(feats[bi * B:(bi + 1) * B], target[bi * B:(bi + 1) * B],
                     lr_at(step, steps, args.lr, args.lr_min), loss=loss)
        if step % args.log_every == 0 or step == steps - 1:
            log.append((step, float(loss[0].item())))
        if args.checkpoint and (step + 1) % args.checkpoint_every == 0:
            save_training_state(args.checkpoint, L, step + 1, {"steps": steps, "frames": N, "seed": args.seed})
    L.sync()
    t_train = time.time() - t2
    params = L.get_params()
    del feats, target
    # held-out evaluation on independent frames
    rf_ho = torch.from_numpy(held_out_frames(w, args.held_out, workers=args.workers)).cuda()
    L.close()
    Le = pam.Learned.from_workload(w, max_frames=args.held_out)
    Le.set_params(params)
    plan = pam.Plan.from_workload(w, max_frames=args.held_out)
    rows = evaluate(Le, plan, rf_ho, w, args.gate_tol)
    meta = {
        "workload": w.name, "frames": N, "epochs": args.epochs, "batch": B, "steps": steps, "lr": args.lr,
        "lr_min": args.lr_min, "bank_sources": args.bank, "seed": args.seed,
        "seconds": {"bank": round(t_bank, 1), "examples": round(t_data, 1), "train": round(t_train, 1)},
        "loss_log": log[:: max(1, len(log) // 40)] + [log[-1]],
        "held_out": summarize(rows), "gate_tol": args.gate_tol,
    }
    save_checkpoint(args.out, params, meta)
    print(json.dumps(meta))
    plan.close()
    Le.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--frames", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-min", type=float, default=5e-5)
    ap.add_argument("--bank", type=int, default=1024, help="single-source responses in the bank")
    ap.add_argument("--gen-batch", type=int, default=256, help="frames per example call")
    ap.add_argument("--held-out", type=int, default=64)
    ap.add_argument("--gate-tol", type=float, default=0.25)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--log-every", type=int, default=100)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--out", default=CHECKPOINT)
    ap.add_argument("--checkpoint", default="", help="training-state file written every --checkpoint-every steps")
    ap.add_argument("--checkpoint-every", type=int, default=500)
    ap.add_argument("--resume", default="", help="training-state file to continue from")
    train(ap.parse_args())


if __name__ == "__main__":
    main()
