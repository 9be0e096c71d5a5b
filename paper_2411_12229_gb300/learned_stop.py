"""Learned early termination of the search (not in the paper).

A 16 -> 64 -> 64 -> 1 MLP reads the search state every `every` expansions
and predicts whether the result set already holds everything the full
fixed-ef search would return.  Training data are traces of the plain search
(``sqg_search_trace``): features at every evaluation point plus the number
of true top-k ids found so far.  A row is labelled 1 when that count already
equals the count at the end of the full search -- stopping there loses no
recall against the fixed-ef search, which stays the fallback cap.

Training runs on the GPU with the library's own kernels (``sqg_mlp_grad``,
``sqg_mlp_adam``); the stop itself is fused into the search kernel.
"""

from __future__ import annotations

import ctypes as C
import dataclasses
import json

import numpy as np
import torch

from . import _binding as B


@dataclasses.dataclass
class StopModel:
    params: torch.Tensor   # SQG_MLP_NPARAM fp32 on the device
    logit: float           # stop when the network's logit exceeds this
    every: int             # evaluation period in expansions
    ef_cap: int            # fixed-ef fallback cap used with the stop
    info: dict


def _sp(stream=None) -> int:
    return int((stream or torch.cuda.current_stream()).cuda_stream)


def collect(ix, queries: np.ndarray, gt: np.ndarray, k: int, ef_cap: int, every: int, chunk: int = 8192,
            target_hits: np.ndarray | None = None, label: str = "final"):
    """Features and labels from traces of the plain search at ef_cap.

    label "all": a row is positive once the result holds all k true
    nearest neighbours (nothing the search could still add would raise its
    recall).  label "final": once it holds as many true top-k ids as
    `target_hits` (per query; default: what the traced search ends with)."""
    cap = max(1, (4 * ef_cap + 64) // every + 1)
    feats, labels, qidx = [], [], []
    gt_d = torch.from_numpy(np.ascontiguousarray(gt[:, :k], dtype=np.int32)).cuda()
    for a in range(0, queries.shape[0], chunk):
        b = min(queries.shape[0], a + chunk)
        qd = torch.from_numpy(np.ascontiguousarray(queries[a:b])).cuda()
        ids, _, st, f, h, n = ix.search_trace(qd, k, ef_cap, gt_d[a:b], cap, stop_every=every)
        ids = ids.cpu().numpy()
        f, h, n = f.cpu().numpy(), h.cpu().numpy(), n.cpu().numpy()
        for i in range(b - a):
            final = len(np.intersect1d(ids[i], gt[a + i, :k]))
            if label == "all":
                final = k
            elif target_hits is not None:
                final = min(final, int(target_hits[a + i]))
            m = n[i]
            if m == 0:
                continue
            feats.append(f[i, :m])
            labels.append((h[i, :m] >= final).astype(np.float32))
            qidx.append(np.full(m, a + i, dtype=np.int32))
    return np.concatenate(feats), np.concatenate(labels), np.concatenate(qidx)


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialized weights, zero biases (flat layout of include/sqg.h)."""
    g = np.random.default_rng(seed)
    W1 = g.standard_normal((64, 16)) * np.sqrt(2 / 16)
    W2 = g.standard_normal((64, 64)) * np.sqrt(2 / 64)
    W3 = g.standard_normal(64) * np.sqrt(1 / 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3, [0.0]]).astype(np.float32)


def grad(params: torch.Tensor, x: torch.Tensor, y: torch.Tensor, w: torch.Tensor, stream=None):
    """(loss, gradient) of the weighted BCE through sqg_mlp_grad."""
    g = torch.empty(B.MLP_NPARAM, device=params.device)
    loss = torch.empty(1, device=params.device)
    scratch = torch.empty(1, device=params.device)
    B.check(B.lib().sqg_mlp_grad(params.data_ptr(), x.data_ptr(), y.data_ptr(), w.data_ptr(), x.shape[0],
                                 g.data_ptr(), loss.data_ptr(), scratch.data_ptr(), _sp(stream)), "sqg_mlp_grad")
    return loss, g


def adam(params, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
    B.check(B.lib().sqg_mlp_adam(params.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), step,
                                 C.c_float(lr), C.c_float(b1), C.c_float(b2), C.c_float(eps), _sp(stream)),
            "sqg_mlp_adam")


def forward(params: torch.Tensor, x: torch.Tensor, stream=None) -> torch.Tensor:
    z = torch.empty(x.shape[0], device=x.device)
    B.check(B.lib().sqg_mlp_forward(params.data_ptr(), x.data_ptr(), x.shape[0], z.data_ptr(), _sp(stream)),
            "sqg_mlp_forward")
    return z


def save_model(path, model: StopModel) -> None:
    """The stop network in a file of its own: weights, threshold, period,
    fixed-ef cap and the training record."""
    np.savez(path, params=model.params.detach().cpu().numpy().astype(np.float32), logit=np.float32(model.logit),
             every=np.int32(model.every), ef_cap=np.int32(model.ef_cap), info=json.dumps(model.info, default=str))


def load_model(path, device=None) -> StopModel:
    with np.load(path, allow_pickle=False) as z:
        params = z["params"]
        if params.shape != (B.MLP_NPARAM,) or params.dtype != np.float32:
            raise ValueError(f"{path}: not a stop network ({params.shape}, {params.dtype})")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        return StopModel(torch.from_numpy(params.copy()).to(dev), float(z["logit"]), int(z["every"]),
                         int(z["ef_cap"]), json.loads(str(z["info"])))


def save_train_state(path, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int, seed: int) -> None:
    """Adam's state after `step` steps, to resume training from."""
    np.savez(path, params=params.cpu().numpy(), m=m.cpu().numpy(), v=v.cpu().numpy(), step=np.int64(step),
             seed=np.int64(seed))


def load_train_state(path) -> dict:
    with np.load(path, allow_pickle=False) as z:
        return {k: z[k].copy() for k in ("params", "m", "v")} | {"step": int(z["step"]), "seed": int(z["seed"])}


def train(feats: np.ndarray, labels: np.ndarray, *, steps: int = 3000, batch: int = 8192, lr: float = 3e-3,
          seed: int = 0, log=None, resume: str | None = None, checkpoint: str | None = None,
          stop_after: int | None = None) -> torch.Tensor:
    """Minibatch Adam on the GPU; classes balanced by sample weights.

    Step t draws its minibatch from a generator seeded with (seed, t), so a
    run resumed from a state file (`resume`, written by `checkpoint`) sees
    the batches the uninterrupted run would; `stop_after` ends the run
    after that many steps (the learning-rate schedule still follows
    `steps`)."""
    dev = torch.device("cuda")
    X = torch.from_numpy(np.ascontiguousarray(feats, dtype=np.float32)).to(dev)
    Y = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.float32)).to(dev)
    pos = float(labels.mean())
    wpos, wneg = 0.5 / max(pos, 1e-6), 0.5 / max(1 - pos, 1e-6)
    W = torch.where(Y > 0.5, torch.tensor(wpos, device=dev), torch.tensor(wneg, device=dev)).float()
    t0 = 0
    if resume is not None:
        st = load_train_state(resume)
        if st["seed"] != seed:
            raise ValueError(f"{resume}: trained with seed {st['seed']}, not {seed}")
        P, m, v = (torch.from_numpy(st[k]).to(dev) for k in ("params", "m", "v"))
        t0 = st["step"]
    else:
        P = torch.from_numpy(init_params(seed)).to(dev)
        m, v = torch.zeros_like(P), torch.zeros_like(P)
    gen = torch.Generator(device=dev)
    n = X.shape[0]
    last = steps if stop_after is None else min(steps, t0 + stop_after)
    for t in range(t0 + 1, last + 1):
        gen.manual_seed(seed * 1_000_003 + t)
        idx = torch.randint(0, n, (min(batch, n),), device=dev, generator=gen)
        loss, g = grad(P, X[idx].contiguous(), Y[idx].contiguous(), W[idx].contiguous())
        adam(P, g, m, v, t, lr * (0.1 if t > 0.8 * steps else 1.0))
        if log and (t % 1000 == 0 or t == steps):
            log(f"stop-mlp step {t}: loss {float(loss):.4f}")
    if checkpoint is not None:
        save_train_state(checkpoint, P, m, v, last, seed)
    return P


def evaluate(ix, queries: torch.Tensor, gt: np.ndarray, k: int, ef: int, model: StopModel | None = None,
             logit: float | None = None, reps: int = 3):
    """(recall, qps, mean hops) of the search with or without the stop."""
    from .eval import recall
    kw = {}
    if model is not None:
        kw = dict(stop_mlp=model.params, stop_logit=model.logit if logit is None else logit,
                  stop_every=model.every)
    ids, _, st = ix.search(queries, k, ef, stats=True, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ix.search(queries, k, ef, **kw)
    e1.record()
    torch.cuda.synchronize()
    qps = reps * queries.shape[0] / (e0.elapsed_time(e1) / 1e3)
    return recall(ids.cpu().numpy(), gt, k), qps, float(st[:, 0].float().mean())


def hits_of(ids: np.ndarray, gt: np.ndarray, k: int) -> np.ndarray:
    return np.array([len(np.intersect1d(ids[i], gt[i, :k])) for i in range(ids.shape[0])], dtype=np.int32)


def fit(ix, train_q: np.ndarray, train_gt: np.ndarray, k: int, ef_cap: int, target: float, *, every: int = 2,
        ef_ref: int | None = None, val_frac: float = 0.2, steps: int = 3000, seed: int = 0, log=None,
        label: str = "final") -> StopModel:
    """Trace, train, then pick the stop threshold on held-out queries: the
    most aggressive logit whose recall still reaches `target`.

    label "all" (the target the stop is built for): a row is positive once
    the result holds the true top-k, so a confident stop loses nothing and
    the queries that never get there run to the fixed-ef cap.  label
    "final" with ef_ref: once the traced search (at ef_cap) holds as many
    true top-k ids as the plain search at ef_ref ends with for that query;
    without ef_ref: as many as the traced search itself ends with."""
    nv = max(1, int(train_q.shape[0] * val_frac))
    tq, tg = train_q[nv:], train_gt[nv:]
    vq, vg = train_q[:nv], train_gt[:nv]
    th = None
    if ef_ref is not None and label != "all":
        th = np.empty(tq.shape[0], dtype=np.int32)
        for a in range(0, tq.shape[0], 8192):
            ids, _ = ix.search(torch.from_numpy(np.ascontiguousarray(tq[a:a + 8192])).cuda(), k, ef_ref)
            th[a:a + 8192] = hits_of(ids.cpu().numpy(), tg[a:a + 8192], k)
    f, y, _ = collect(ix, tq, tg, k, ef_cap, every, target_hits=th, label=label)
    P = train(f, y, steps=steps, seed=seed, log=log)
    model = StopModel(P, 0.0, every, ef_cap, dict(rows=int(f.shape[0]), positive=float(y.mean()), label=label))
    vqd = torch.from_numpy(np.ascontiguousarray(vq)).cuda()
    best = None
    for thr in (6.0, 5.0, 4.0, 3.0, 2.0, 1.5, 1.0, 0.5, 0.0, -0.5, -1.0, -2.0):
        r, qps, hops = evaluate(ix, vqd, vg, k, ef_cap, model, logit=thr, reps=2)
        if log:
            log(f"stop threshold {thr:+.1f}: recall {r:.4f} hops {hops:.1f} qps {qps:.0f}")
        if r >= target:
            best = thr
        else:
            break
    model.logit = 6.0 if best is None else best
    model.info.update(threshold=model.logit, val_queries=nv)
    return model


def fit_mixed(ix, train_q: np.ndarray, train_gt: np.ndarray, groups, target, *, every: int = 4,
              val_frac: float = 0.2, steps: int = 3000, seed: int = 0, log=None,
              max_loss: float | None = None) -> StopModel:
    """One stop network for requests of several k (the serving workload's
    k in {10, 100}): groups = [(k, ef_cap), ...].  Traces of every group
    are pooled with the label "the result holds the true top-k" (the
    features carry k, so the network can tell the groups apart); the
    threshold is the most aggressive logit whose held-out recall@10 reaches
    `target` in every group (a float, or a {k: target} dict; with max_loss,
    the plain search's held-out recall at each group's cap minus max_loss).
    The model's ef_cap is the largest group's."""
    from .eval import recall as _recall
    vq0, vg0 = train_q[:max(1, int(train_q.shape[0] * val_frac))], train_gt[:max(1, int(train_q.shape[0] * val_frac))]
    if max_loss is not None:
        vqd0 = torch.from_numpy(np.ascontiguousarray(vq0)).cuda()
        tgt = {}
        for k, cap in groups:
            ids, _ = ix.search(vqd0, k, cap)
            kk = min(k, 10)
            tgt[k] = _recall(ids.cpu().numpy()[:, :kk], vg0, kk) - max_loss
    else:
        tgt = target if isinstance(target, dict) else {k: target for k, _ in groups}
    nv = max(1, int(train_q.shape[0] * val_frac))
    tq, tg = train_q[nv:], train_gt[nv:]
    vq, vg = train_q[:nv], train_gt[:nv]
    fs, ys = [], []
    for k, cap in groups:
        f, y, _ = collect(ix, tq, tg, k, cap, every, label="all")
        fs.append(f)
        ys.append(y)
    f, y = np.concatenate(fs), np.concatenate(ys)
    P = train(f, y, steps=steps, seed=seed, log=log)
    model = StopModel(P, 0.0, every, max(c for _, c in groups),
                      dict(rows=int(f.shape[0]), positive=float(y.mean()), label="all", groups=list(groups)))
    vqd = torch.from_numpy(np.ascontiguousarray(vq)).cuda()
    best = None
    for thr in (6.0, 5.0, 4.0, 3.0, 2.0, 1.5, 1.0, 0.5, 0.0, -0.5, -1.0, -2.0):
        ok = True
        for k, cap in groups:
            ids, _ = ix.search(vqd, k, cap, stop_mlp=P, stop_logit=thr, stop_every=every)
            from .eval import recall
            kk = min(k, 10)
            r = recall(ids.cpu().numpy()[:, :kk], vg, kk)
            ok = ok and r >= tgt[k]
            if log:
                log(f"stop threshold {thr:+.1f} k={k} ef={cap}: recall@10 {r:.4f}")
        if not ok:
            break
        best = thr
    model.logit = 6.0 if best is None else best
    model.info.update(threshold=model.logit, val_queries=nv)
    return model


def perfect_stop(ix, queries: np.ndarray, gt: np.ndarray, k: int, ef_cap: int, chunk: int = 4096) -> dict:
    """What any stop can gain at this cap: traces of the plain search
    (features after every expansion once the result holds k entries) give,
    per query, the first expansion after which the result holds all k true
    nearest neighbours.  A stop that fired exactly there, and never for
    queries that do not get there, keeps the plain search's recall and
    expands min(that expansion, the plain count).  Returns the plain recall
    and mean expansions and this bound's mean expansions."""
    from .eval import recall
    cap = 4 * ef_cap + 64
    gt_d = torch.from_numpy(np.ascontiguousarray(gt[:, :k], dtype=np.int32)).cuda()
    hops_all, best_all, ids_all = [], [], []
    for a in range(0, queries.shape[0], chunk):
        b = min(queries.shape[0], a + chunk)
        qd = torch.from_numpy(np.ascontiguousarray(queries[a:b])).cuda()
        ids, _, st, f, h, n = ix.search_trace(qd, k, ef_cap, gt_d[a:b], cap, stop_every=1)
        hops = st[:, 0].cpu().numpy().astype(np.int64)
        f0 = f[:, :, 0].cpu().numpy()  # hops / ef at each evaluation point
        h, n = h.cpu().numpy(), n.cpu().numpy()
        for i in range(b - a):
            rows = np.nonzero(h[i, :n[i]] >= k)[0]
            best_all.append(int(round(float(f0[i, rows[0]]) * ef_cap)) if rows.size else int(hops[i]))
        hops_all.append(hops)
        ids_all.append(ids.cpu().numpy())
    hops = np.concatenate(hops_all)
    best = np.minimum(np.array(best_all, dtype=np.int64), hops)
    return {"ef": int(ef_cap), "recall": round(recall(np.concatenate(ids_all), gt, k), 4),
            "hops": round(float(hops.mean()), 2), "perfect_stop_hops": round(float(best.mean()), 2),
            "saving": round(1.0 - float(best.mean()) / float(hops.mean()), 4)}
