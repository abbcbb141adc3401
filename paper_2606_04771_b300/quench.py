"""Quench driver: the open Fermi-Hubbard chain from the Neel state (Eq. neel) evolved
with TDVP (Sec. S2.2) to a final time, one JSON line per time step.

    python -m paper_2606_04771_b300.quench --L 60 --U 4 --dt 0.05 --t 3 --chi 4096 \
        --eps 1e-9 --mode adaptive --precision bf16x4 --out run.npz
    python -m paper_2606_04771_b300.quench --L 31 --vacancy --symmetry u1u1 ...
    python -m paper_2606_04771_b300.quench ... --checkpoint run.ckpt --checkpoint-every 20
    python -m paper_2606_04771_b300.quench --resume run.ckpt --t 6 ...

Every step prints t, the integrator used, the largest bond dimension (U(1)-equivalent
and reduced) and every bond's, the largest discarded weight and Krylov dimension so
far, the seconds and H_eff TFLOP/s of the step and the device memory held.  Every
--measure-every steps (and at the end) it also measures n_i, S^z_i, docc_i, the
energy and (with --entropy) every bond's entanglement entropy, and stores them in
--out (numpy .npz: t, n_up, n_dn, docc, s_ent, energy).
All arithmetic runs in the CUDA library; this module only drives it.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from ._lib import Chain, vacancy_occupations


def run(L=60, J=1.0, U=4.0, dt=0.05, t_final=3.0, chi=4096, eps=1e-9, mode="adaptive", precision="bf16x4",
        symmetry="su2", measure_every=10, entropy=True, out=None, stream=None, log=sys.stdout, vacancy=False,
        checkpoint=None, checkpoint_every=0, resume=None):
    """checkpoint: file written every checkpoint_every steps (if > 0) and at the end;
    resume: a checkpoint to continue from (its chain replaces L, J, U, symmetry and
    the initial state; the run goes on from its stored time to t_final)."""
    k0 = 0
    if resume:
        ch, t_start = Chain.load(resume, precision=precision, stream=stream)
        L = ch.L
        k0 = int(round(t_start / dt))
    else:
        ch = Chain(L, J, U, symmetry=symmetry, precision=precision, stream=stream,
                   occupations=vacancy_occupations(L) if vacancy else None)
    nsteps = int(round(t_final / dt))
    rec = {"t": [], "n_up": [], "n_dn": [], "docc": [], "s_ent": [], "energy": []}
    t0 = time.perf_counter()

    def measure(t):
        o = ch.measure(entropy=entropy, energy=True)
        rec["t"].append(t)
        for k in ("n_up", "n_dn", "docc"):
            rec[k].append(o[k])
        rec["s_ent"].append(o["s_ent"] if entropy else np.zeros(L - 1))
        rec["energy"].append(o["energy"])
        return o

    measure(k0 * dt)
    flops0 = ch.stats()["heff_flops"]
    for k in range(k0 + 1, nsteps + 1):
        ts = time.perf_counter()
        used = ch.step(dt, chi, eps, mode=mode)
        sec = time.perf_counter() - ts
        chis, red = ch.bond_dims()
        st = ch.stats()
        line = {"step": k, "t": round(k * dt, 10), "mode": used, "chi": int(chis.max()), "chi_red": int(red.max()),
                "max_discarded": st["max_discarded"], "max_krylov": int(st["max_krylov"]), "seconds": sec,
                "heff_tflops": (st["heff_flops"] - flops0) / sec / 1e12, "elapsed": time.perf_counter() - t0,
                "device_gb": st["device_bytes"] / 1e9, "chi_bonds": chis.tolist()}
        flops0 = st["heff_flops"]
        if k % measure_every == 0 or k == nsteps:
            o = measure(k * dt)
            line.update({"energy": o["energy"], "n_up_mid": float(o["n_up"][L // 2]),
                         "docc_mean": float(np.mean(o["docc"]))})
            if entropy:
                line["s_half"] = float(o["s_ent"][L // 2 - 1])
        if checkpoint and ((checkpoint_every > 0 and k % checkpoint_every == 0) or k == nsteps):
            ch.save(checkpoint, t=k * dt)
            line["checkpoint"] = checkpoint
        if log is not None:
            print(json.dumps(line), file=log, flush=True)
    ch.close()
    res = {k: np.array(v) for k, v in rec.items()}
    if out:
        np.savez(out, **res)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=60)
    ap.add_argument("--J", type=float, default=1.0)
    ap.add_argument("--U", type=float, default=4.0)
    ap.add_argument("--dt", type=float, default=0.05)
    ap.add_argument("--t", type=float, default=3.0)
    ap.add_argument("--chi", type=int, default=4096)
    ap.add_argument("--eps", type=float, default=1e-9)
    ap.add_argument("--mode", default="adaptive", choices=["two", "one", "adaptive"])
    ap.add_argument("--precision", default="bf16x4", choices=["fp64", "3xtf32", "bf16x4"])
    ap.add_argument("--symmetry", default="su2", choices=["su2", "u1u1"])
    ap.add_argument("--measure-every", type=int, default=10)
    ap.add_argument("--entropy", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("--vacancy", action="store_true", help="Neel state with the centre site empty (use u1u1)")
    ap.add_argument("--checkpoint", default=None, help="checkpoint file, written at the end and every --checkpoint-every")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default=None, help="continue from this checkpoint to --t")
    a = ap.parse_args(argv)
    run(a.L, a.J, a.U, a.dt, a.t, a.chi, a.eps, a.mode, a.precision, a.symmetry, a.measure_every, a.entropy, a.out,
        vacancy=a.vacancy, checkpoint=a.checkpoint, checkpoint_every=a.checkpoint_every, resume=a.resume)


if __name__ == "__main__":
    main()
