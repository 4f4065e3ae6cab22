"""Thin ctypes binding of the Pasur GB300 C ABI (include/pasur.h).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libpasur.so``.  There is no CPU fallback: if the library is missing or no CUDA device is
present, the calls raise.  Arrays may be numpy arrays (host) or torch CUDA tensors (device); the
library detects which.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpasur.so")

PASUR_OK, PASUR_EINVAL, PASUR_ENOMEM, PASUR_EOVERFLOW = 0, -1, -2, -3
PASUR_ECUDA, PASUR_ETIMEOUT, PASUR_ENUMERIC, PASUR_ENOTIMPL = -4, -5, -6, -7
_NAMES = {0: "PASUR_OK", -1: "PASUR_EINVAL", -2: "PASUR_ENOMEM", -3: "PASUR_EOVERFLOW", -4: "PASUR_ECUDA",
          -5: "PASUR_ETIMEOUT", -6: "PASUR_ENUMERIC", -7: "PASUR_ENOTIMPL"}

# every symbol the header declares (checked by the CPU test suite)
EXPORTS = [
    "pasur_config_default", "pasur_create", "pasur_destroy", "pasur_last_error", "pasur_memory", "pasur_launch_count",
    "pasur_deal",
    "pasur_build_round", "pasur_tree_free", "pasur_tree_sizes", "pasur_unfold", "pasur_cfr_iterate",
    "pasur_avg_strategy", "pasur_round_utilities", "pasur_next_roots", "pasur_export_level", "pasur_leaf_values",
    "pasur_last_cfr_stats", "pasur_batch_create", "pasur_batch_solve", "pasur_batch_tree", "pasur_batch_stats",
    "pasur_batch_free", "pasur_move_offsets_noalloc", "pasur_selfplay", "pasur_batch_selfplay",
    "pasur_last_selfplay_stats", "pasur_mlp_create", "pasur_mlp_free", "pasur_mlp_set_params", "pasur_mlp_get_params",
    "pasur_mlp_forward", "pasur_mlp_gradients", "pasur_mlp_dataset_add_tree", "pasur_mlp_dataset_add_rows",
    "pasur_mlp_dataset_size", "pasur_mlp_dataset_export", "pasur_mlp_dataset_clear", "pasur_mlp_train",
    "pasur_mlp_predict_next", "pasur_mlp_root_features", "pasur_mlp_stats", "pasur_root_values",
    "pasur_batch_create_cut", "pasur_solved_sizes", "pasur_batch_work", "pasur_cfr_convergence",
    "pasur_root_paths", "pasur_cfr_iterate_roots", "pasur_root_sizes", "pasur_round_reach",
    "pasur_batch_create_roots", "pasur_batch_set_cut_values", "pasur_swept_pairs", "pasur_batch_pairs",
    "pasur_save_round", "pasur_load_round", "pasur_avg_strategy_async", "pasur_sync", "pasur_response_reach",
]


class PasurError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class pasur_score(C.Structure):
    _fields_ = [("a_clubs", C.c_int16), ("b_clubs", C.c_int16), ("delta", C.c_int16), ("bonus", C.c_int16)]


class pasur_config(C.Structure):
    _fields_ = [("variant", C.c_int32), ("iters", C.c_int32), ("rm_deadzone", C.c_float), ("dcfr_alpha", C.c_float),
                ("dcfr_beta", C.c_float), ("dcfr_gamma", C.c_float), ("slots_per_item", C.c_int32),
                ("threads", C.c_int32), ("split_bytes", C.c_int32), ("stream_bytes", C.c_int32),
                ("merge_delta", C.c_int32)]


_lib = None
vp = C.c_void_p
i64 = C.c_int64
i64p = C.POINTER(C.c_int64)


def load() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"Pasur CUDA library not built ({LIB_PATH}); run paper_2508_06559_gb300/build.py")
    L = C.CDLL(LIB_PATH)
    L.pasur_config_default.argtypes = [C.POINTER(pasur_config)]
    L.pasur_create.argtypes = [C.POINTER(vp), C.c_int, C.c_size_t, vp]
    L.pasur_destroy.argtypes = [vp]
    L.pasur_last_error.argtypes = [vp]
    L.pasur_last_error.restype = C.c_char_p
    L.pasur_memory.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    L.pasur_launch_count.argtypes = [vp, i64p]
    L.pasur_deal.argtypes = [C.c_uint64, vp]
    L.pasur_build_round.argtypes = [vp, vp, C.c_int, vp, i64, C.POINTER(vp)]
    L.pasur_tree_free.argtypes = [vp]
    L.pasur_tree_sizes.argtypes = [vp, vp, vp]
    L.pasur_unfold.argtypes = [vp, vp, vp, vp]
    L.pasur_cfr_iterate.argtypes = [vp, C.POINTER(pasur_config), vp]
    L.pasur_avg_strategy.argtypes = [vp, vp, i64]
    L.pasur_round_utilities.argtypes = [vp, vp, i64]
    L.pasur_next_roots.argtypes = [vp, vp, i64, vp, vp, i64, vp, i64p, i64p]
    L.pasur_export_level.argtypes = [vp, C.c_int, i64, vp, vp, vp, vp, vp, vp]
    L.pasur_leaf_values.argtypes = [vp, vp, i64]
    L.pasur_last_cfr_stats.argtypes = [vp, C.POINTER(C.c_float), i64p, C.POINTER(C.c_int32)]
    L.pasur_solved_sizes.argtypes = [vp, vp, i64p]
    L.pasur_batch_work.argtypes = [vp, i64p, i64p]
    L.pasur_swept_pairs.argtypes = [vp, i64p]
    L.pasur_save_round.argtypes = [vp, vp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.pasur_load_round.argtypes = [vp, vp, C.c_size_t]
    L.pasur_avg_strategy_async.argtypes = [vp, vp, i64]
    L.pasur_sync.argtypes = [vp]
    L.pasur_response_reach.argtypes = [vp, C.c_int, vp, vp, vp, vp, i64]
    L.pasur_batch_pairs.argtypes = [vp, i64p]
    L.pasur_root_paths.argtypes = [vp, vp, i64]
    L.pasur_cfr_iterate_roots.argtypes = [vp, C.POINTER(pasur_config), vp, i64, i64]
    L.pasur_root_sizes.argtypes = [vp, vp, i64]
    L.pasur_round_reach.argtypes = [vp, vp, vp, vp, i64]
    L.pasur_batch_create_roots.argtypes = [vp, vp, i64, C.c_int, vp, vp, vp, vp, C.POINTER(pasur_config), C.POINTER(vp)]
    L.pasur_batch_set_cut_values.argtypes = [vp, i64, vp, i64]
    L.pasur_cfr_convergence.argtypes = [vp, C.POINTER(pasur_config), vp, vp, C.c_int, vp]
    L.pasur_move_offsets_noalloc.argtypes = [vp, i64, vp, vp]
    L.pasur_batch_create.argtypes = [vp, vp, i64, C.c_int, C.POINTER(pasur_config), C.POINTER(vp)]
    L.pasur_batch_create_cut.argtypes = [vp, vp, i64, C.c_int, C.c_int, C.POINTER(pasur_config), vp, C.POINTER(vp)]
    L.pasur_batch_solve.argtypes = [vp, vp, i64]
    L.pasur_batch_tree.argtypes = [vp, i64, C.c_int, C.POINTER(vp)]
    L.pasur_batch_stats.argtypes = [vp, C.POINTER(C.c_float), i64p, i64p]
    L.pasur_batch_free.argtypes = [vp]
    L.pasur_selfplay.argtypes = [vp, C.POINTER(vp), C.c_int, C.POINTER(vp), i64, i64, C.c_uint64, vp]
    L.pasur_batch_selfplay.argtypes = [vp, i64, vp, vp]
    L.pasur_last_selfplay_stats.argtypes = [vp, C.POINTER(C.c_float), i64p]
    L.pasur_root_values.argtypes = [vp, C.c_int, vp, vp, vp, i64]
    L.pasur_mlp_create.argtypes = [vp, i64, C.c_uint64, C.POINTER(vp)]
    L.pasur_mlp_free.argtypes = [vp]
    L.pasur_mlp_set_params.argtypes = [vp, vp, i64]
    L.pasur_mlp_get_params.argtypes = [vp, vp, i64]
    L.pasur_mlp_forward.argtypes = [vp, vp, i64, vp]
    L.pasur_mlp_gradients.argtypes = [vp, vp, vp, i64, vp, vp]
    L.pasur_mlp_dataset_add_tree.argtypes = [vp, vp]
    L.pasur_mlp_dataset_add_rows.argtypes = [vp, vp, vp, i64]
    L.pasur_mlp_dataset_size.argtypes = [vp, i64p]
    L.pasur_mlp_dataset_export.argtypes = [vp, i64, i64, vp, vp]
    L.pasur_mlp_dataset_clear.argtypes = [vp]
    L.pasur_mlp_train.argtypes = [vp, C.c_int, i64, C.c_float, C.c_uint64, vp]
    L.pasur_mlp_predict_next.argtypes = [vp, vp, vp, i64]
    L.pasur_mlp_root_features.argtypes = [vp, vp, C.c_int, vp, vp, vp, i64, vp]
    L.pasur_mlp_stats.argtypes = [vp, C.POINTER(C.c_float), i64p]
    for name in EXPORTS:
        if name != "pasur_last_error":
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def _check(rc: int, ctx_handle=None):
    if rc != PASUR_OK:
        msg = load().pasur_last_error(ctx_handle)
        raise PasurError(rc, msg.decode() if msg else "")


def pasur_config_default(**over) -> pasur_config:
    cfg = pasur_config()
    _check(load().pasur_config_default(C.byref(cfg)))
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def pasur_deal(seed: int) -> np.ndarray:
    deck = np.zeros(52, np.uint8)
    _check(load().pasur_deal(C.c_uint64(seed), _ptr(deck)))
    return deck


def pasur_move_offsets_noalloc(counts_dev, offsets_dev, stream=None) -> None:
    """CSR offsets (n+1 int64, device) from per-node move counts (n int32, device) without any
    device allocation; see include/pasur.h.  counts_dev: contiguous CUDA int32 tensor of n counts;
    offsets_dev: contiguous CUDA int64 tensor of at least n+1 elements on the same device (the C
    call cannot check its length, so this wrapper does).  stream: a cudaStream_t handle, default
    torch's current stream on that device (the stream the tensors' producers normally used).
    Raises PasurError (PASUR_EINVAL for a wrong tensor) on failure."""
    import torch

    def bad(msg):
        raise PasurError(PASUR_EINVAL, "pasur_move_offsets_noalloc: " + msg)

    for name, t, dt in (("counts", counts_dev, torch.int32), ("offsets", offsets_dev, torch.int64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            bad(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            bad(f"{name} must be {dt}, not {t.dtype}")
        if not t.is_contiguous():
            bad(f"{name} must be contiguous")
    if counts_dev.device != offsets_dev.device:
        bad("counts and offsets must be on the same device")
    n = counts_dev.numel()
    if offsets_dev.numel() < n + 1:
        bad(f"offsets holds {offsets_dev.numel()} elements, {n + 1} are written")
    if stream is None:
        stream = torch.cuda.current_stream(counts_dev.device).cuda_stream
    with torch.cuda.device(counts_dev.device):
        _check(load().pasur_move_offsets_noalloc(_ptr(counts_dev), n, _ptr(offsets_dev), stream))


def scores_array(rows) -> np.ndarray:
    """(n,4) int16 rows (a_clubs, b_clubs, delta, bonus) -> contiguous pasur_score array."""
    return np.ascontiguousarray(np.asarray(rows, np.int16).reshape(-1, 4))


class Ctx:
    """pasur_create / pasur_destroy."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None):
        h = vp()
        rc = load().pasur_create(C.byref(h), device, hbm_budget_bytes, stream)
        _check(rc, None)
        self.h = h
        self._trees = weakref.WeakSet()
        self._batches = weakref.WeakSet()

    def close(self):
        """Free the context's remaining trees and batches, then the context."""
        if self.h:
            for t in list(self._trees):
                t.free()
            for b in list(self._batches):
                b.free()
            _check(load().pasur_destroy(self.h), self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pasur_sync(self) -> None:
        """Wait for the context's stream and the copies of asynchronous exports."""
        _check(load().pasur_sync(self.h), self.h)

    def memory(self):
        a, b = C.c_size_t(0), C.c_size_t(0)
        _check(load().pasur_memory(self.h, C.byref(a), C.byref(b)), self.h)
        return a.value, b.value

    def pasur_launch_count(self) -> int:
        n = C.c_int64(0)
        _check(load().pasur_launch_count(self.h, C.byref(n)), self.h)
        return n.value

    def pasur_build_round(self, deck, rnd: int, root_pools) -> "Tree":
        d = np.ascontiguousarray(deck, np.uint8)
        pools = root_pools if hasattr(root_pools, "data_ptr") else np.ascontiguousarray(root_pools, np.uint64)
        n = pools.numel() if hasattr(pools, "numel") else len(pools)
        th = vp()
        _check(load().pasur_build_round(self.h, _ptr(d), rnd, _ptr(pools), n, C.byref(th)), self.h)
        t = Tree(self, th)
        self._trees.add(t)
        return t


    def pasur_selfplay(self, trees, n_games: int, seed: int, root_q: int = 0, sigmas=None, out=None):
        """Final game differences (int16 per game) of sampled games through consecutive round
        trees; sigmas: None, or per round None (the tree's average strategy) or a float32 array
        or tensor per FGT edge."""
        hs = (vp * len(trees))(*[t.h for t in trees])
        keep = []
        sp = None
        if sigmas is not None:
            ptrs = []
            for sg in sigmas:
                if sg is None:
                    ptrs.append(None)
                else:
                    sg = sg if hasattr(sg, "data_ptr") else np.ascontiguousarray(sg, np.float32)
                    keep.append(sg)
                    ptrs.append(_ptr(sg))
            sp = (vp * len(ptrs))(*ptrs)
        if out is None:
            out = np.zeros(n_games, np.int16)
        _check(load().pasur_selfplay(self.h, hs, len(trees), sp, root_q, n_games, seed, _ptr(out)), self.h)
        return out

    def pasur_last_selfplay_stats(self):
        ms, g = C.c_float(0), C.c_int64(0)
        _check(load().pasur_last_selfplay_stats(self.h, C.byref(ms), C.byref(g)), self.h)
        return ms.value, g.value


N_MLP_PARAMS = 3 * 256 * 256 + 3 * 256 + 256 + 1


class Mlp:
    """The round-start utility surrogate (pasur_mlp_*).  Feature rows are bf16 bit patterns
    (uint16 [n, 256])."""

    def __init__(self, ctx: "Ctx", dataset_capacity: int = 0, seed: int = 0):
        h = vp()
        _check(load().pasur_mlp_create(ctx.h, dataset_capacity, seed, C.byref(h)), ctx.h)
        self.ctx, self.h = ctx, h
        ctx._batches.add(self)

    def free(self):
        if self.h and self.ctx.h:
            load().pasur_mlp_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _c(self, rc):
        _check(rc, self.ctx.h)

    def set_params(self, flat):
        f = np.ascontiguousarray(flat, np.float32)
        self._c(load().pasur_mlp_set_params(self.h, _ptr(f), f.size))

    def get_params(self) -> np.ndarray:
        out = np.zeros(N_MLP_PARAMS, np.float32)
        self._c(load().pasur_mlp_get_params(self.h, _ptr(out), out.size))
        return out

    def forward(self, x, out=None):
        x = x if hasattr(x, "data_ptr") else np.ascontiguousarray(x, np.uint16)
        n = x.shape[0]
        if out is None:
            out = np.zeros(n, np.float32)
        self._c(load().pasur_mlp_forward(self.h, _ptr(x), n, _ptr(out)))
        return out

    def gradients(self, x, y):
        x = np.ascontiguousarray(x, np.uint16)
        y = np.ascontiguousarray(y, np.float32)
        loss = np.zeros(1, np.float32)
        g = np.zeros(N_MLP_PARAMS, np.float32)
        self._c(load().pasur_mlp_gradients(self.h, _ptr(x), _ptr(y), len(y), _ptr(loss), _ptr(g)))
        return float(loss[0]), g

    def dataset_add_tree(self, tree: "Tree"):
        self._c(load().pasur_mlp_dataset_add_tree(self.h, tree.h))

    def dataset_add_rows(self, x, y):
        x = x if hasattr(x, "data_ptr") else np.ascontiguousarray(x, np.uint16)
        y = y if hasattr(y, "data_ptr") else np.ascontiguousarray(y, np.float32)
        self._c(load().pasur_mlp_dataset_add_rows(self.h, _ptr(x), _ptr(y), x.shape[0]))

    def dataset_size(self) -> int:
        n = C.c_int64(0)
        self._c(load().pasur_mlp_dataset_size(self.h, C.byref(n)))
        return n.value

    def dataset_export(self, first: int = 0, count=None):
        if count is None:
            count = self.dataset_size() - first
        x = np.zeros((count, 256), np.uint16)
        y = np.zeros(count, np.float32)
        self._c(load().pasur_mlp_dataset_export(self.h, first, count, _ptr(x), _ptr(y)))
        return x, y

    def dataset_clear(self):
        self._c(load().pasur_mlp_dataset_clear(self.h))

    def train(self, epochs: int, batch: int, lr: float, shuffle_seed: int = 0) -> np.ndarray:
        losses = np.zeros(max(epochs, 1), np.float32)
        self._c(load().pasur_mlp_train(self.h, epochs, batch, lr, shuffle_seed, _ptr(losses)))
        return losses[:epochs]

    def predict_next(self, tree: "Tree", out=None):
        n = tree.n_next_roots()
        if out is None:
            out = np.zeros(n, np.float32)
        cap = out.numel() if hasattr(out, "numel") else len(out)
        self._c(load().pasur_mlp_predict_next(self.h, tree.h, _ptr(out), cap))
        return out

    def stats(self):
        ms, st = C.c_float(0), C.c_int64(0)
        self._c(load().pasur_mlp_stats(self.h, C.byref(ms), C.byref(st)))
        return ms.value, st.value


def pasur_mlp_root_features(ctx: "Ctx", deck, rnd: int, pools, score_offs, scores) -> np.ndarray:
    d = np.ascontiguousarray(deck, np.uint8)
    p = np.ascontiguousarray(pools, np.uint64)
    so = np.ascontiguousarray(score_offs, np.int64)
    sc = scores_array(scores)
    out = np.zeros((int(so[-1]), 256), np.uint16)
    _check(load().pasur_mlp_root_features(ctx.h, _ptr(d), rnd, _ptr(p), _ptr(so), _ptr(sc), len(p), _ptr(out)), ctx.h)
    return out


def chain_values(trees, mode: int, sigmas=None) -> np.ndarray:
    """Root values of trees[0] with every round's leaves linked to the next tree's values
    (trees: consecutive rounds ending with the final one; sigmas: per round or None)."""
    nxt = None
    for i in range(len(trees) - 1, -1, -1):
        nxt = trees[i].pasur_root_values(mode, None if sigmas is None else sigmas[i], nxt)
    return nxt


class Batch:
    """pasur_batch_create / _solve / _tree / _stats / _free: many deals solved together."""

    def __init__(self, ctx: Ctx, decks, first_round: int, cfg: pasur_config, last_round: int = 5, mlp=None, roots=None):
        """roots: None, or per deal (pools, score offsets, scores) of its first round
        (pasur_batch_create_roots)."""
        d = np.ascontiguousarray(np.asarray(decks, np.uint8).reshape(-1, 52))
        h = vp()
        if roots is not None:
            dr, pl, so, sc = [0], [], [0], []
            for pools, soff, scores in roots:
                pools = np.asarray(pools, np.uint64)
                soff = np.asarray(soff, np.int64)
                scores = np.asarray(scores, np.int16).reshape(-1, 4)
                pl.append(pools)
                base = so[-1]
                so.extend((base + soff[1:]).tolist())
                sc.append(scores)
                dr.append(dr[-1] + len(pools))
            dr = np.array(dr, np.int64)
            pl = np.ascontiguousarray(np.concatenate(pl) if pl else np.zeros(0, np.uint64), np.uint64)
            so = np.array(so, np.int64)
            sc = np.ascontiguousarray(np.concatenate(sc) if sc else np.zeros((0, 4), np.int16), np.int16)
            rc = load().pasur_batch_create_roots(ctx.h, _ptr(d), d.shape[0], first_round, _ptr(dr), _ptr(pl), _ptr(so),
                                                 _ptr(sc), C.byref(cfg), C.byref(h))
        elif last_round == 5 and mlp is None:
            rc = load().pasur_batch_create(ctx.h, _ptr(d), d.shape[0], first_round, C.byref(cfg), C.byref(h))
        else:
            rc = load().pasur_batch_create_cut(ctx.h, _ptr(d), d.shape[0], first_round, last_round, C.byref(cfg),
                                               mlp.h if mlp is not None else None, C.byref(h))
        _check(rc, ctx.h)
        self.ctx, self.h, self.n_deals, self.first_round, self.last_round = ctx, h, d.shape[0], first_round, last_round
        ctx._batches.add(self)

    def free(self):
        if self.h and self.ctx.h:
            load().pasur_batch_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def pasur_batch_solve(self, out=None):
        if out is None:
            out = np.zeros(self.n_deals, np.float32)
        n = out.numel() if hasattr(out, "numel") else len(out)
        _check(load().pasur_batch_solve(self.h, _ptr(out), n), self.ctx.h)
        return out

    def pasur_batch_tree(self, deal: int, rnd: int) -> "Tree":
        th = vp()
        _check(load().pasur_batch_tree(self.h, deal, rnd, C.byref(th)), self.ctx.h)
        return Tree(self.ctx, th, owned=False)

    def pasur_batch_stats(self):
        ms, e, l = C.c_float(0), C.c_int64(0), C.c_int64(0)
        _check(load().pasur_batch_stats(self.h, C.byref(ms), C.byref(e), C.byref(l)), self.ctx.h)
        return ms.value, e.value, l.value

    def pasur_batch_set_cut_values(self, deal: int, values):
        v = values if hasattr(values, "data_ptr") else np.ascontiguousarray(values, np.float32)
        n = v.numel() if hasattr(v, "numel") else len(v)
        _check(load().pasur_batch_set_cut_values(self.h, deal, _ptr(v), n), self.ctx.h)

    def pasur_batch_work(self):
        """(FGT edges over the solved slots, swept edges with CFR state) of one solve."""
        a, b = C.c_int64(0), C.c_int64(0)
        _check(load().pasur_batch_work(self.h, C.byref(a), C.byref(b)), self.ctx.h)
        return a.value, b.value

    def pasur_batch_pairs(self) -> int:
        """(active node, solved slot) pairs updated per iteration, all trees."""
        a = C.c_int64(0)
        _check(load().pasur_batch_pairs(self.h, C.byref(a)), self.ctx.h)
        return a.value

    def pasur_batch_selfplay(self, n_games: int, seeds, out=None):
        """n_games games per deal (deal d under seeds[d]); int16 [n_deals, n_games]."""
        sd = np.ascontiguousarray(seeds, np.uint64)
        assert sd.shape == (self.n_deals,)
        if out is None:
            out = np.zeros((self.n_deals, n_games), np.int16)
        _check(load().pasur_batch_selfplay(self.h, n_games, _ptr(sd), _ptr(out)), self.ctx.h)
        return out


class Tree:
    """One round: wraps the pasur_tree calls (names as in the C ABI)."""

    def __init__(self, ctx: Ctx, h, owned: bool = True):
        self.ctx, self.h, self.owned = ctx, h, owned

    def free(self):
        if self.h and self.ctx.h and self.owned:
            load().pasur_tree_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _c(self, rc):
        _check(rc, self.ctx.h)

    def pasur_tree_sizes(self):
        g = np.zeros(9, np.int64)
        q = np.zeros(9, np.int64)
        self._c(load().pasur_tree_sizes(self.h, _ptr(g), _ptr(q)))
        return g, q

    def pasur_cfr_convergence(self, cfg: pasur_config, checkpoints, next_root_util=None) -> np.ndarray:
        """MSE of the average strategy at each checkpoint (iteration counts) to the last one."""
        cp = np.ascontiguousarray(checkpoints, np.int64)
        out = np.zeros(len(cp), np.float64)
        nu = None
        if next_root_util is not None:
            nu = next_root_util if hasattr(next_root_util, "data_ptr") else np.ascontiguousarray(next_root_util, np.float32)
        self._c(load().pasur_cfr_convergence(self.h, C.byref(cfg), _ptr(nu), _ptr(cp), len(cp), _ptr(out)))
        return out

    def pasur_root_paths(self) -> np.ndarray:
        """Per GT root: 0..4 resident size class, 5 streamed, 6 cluster, -1 no CFR work."""
        n = int(self.pasur_tree_sizes()[0][0])
        out = np.zeros(max(n, 1), np.int32)
        self._c(load().pasur_root_paths(self.h, _ptr(out), n))
        return out[:n]

    def pasur_solved_sizes(self):
        """(solved FGT level sizes [9], swept edges) after the first pasur_cfr_iterate."""
        c = np.zeros(9, np.int64)
        e = C.c_int64(0)
        self._c(load().pasur_solved_sizes(self.h, _ptr(c), C.byref(e)))
        return c, e.value

    def pasur_save_round(self) -> np.ndarray:
        """The round's CFR checkpoint (header, regrets, strategy sums, root-value sums) as bytes."""
        n = C.c_size_t(0)
        self._c(load().pasur_save_round(self.h, None, 0, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        self._c(load().pasur_save_round(self.h, _ptr(buf), n.value, C.byref(n)))
        return buf

    def pasur_load_round(self, buf) -> None:
        b = np.ascontiguousarray(buf, np.uint8)
        self._c(load().pasur_load_round(self.h, _ptr(b), b.nbytes))

    def pasur_swept_pairs(self) -> int:
        """(active node, solved slot) pairs updated per iteration, after the first pasur_cfr_iterate."""
        e = C.c_int64(0)
        self._c(load().pasur_swept_pairs(self.h, C.byref(e)))
        return e.value

    def pasur_unfold(self, score_offs, scores) -> np.ndarray:
        so = np.ascontiguousarray(score_offs, np.int64)
        sc = scores_array(scores)
        q = np.zeros(9, np.int64)
        self._c(load().pasur_unfold(self.h, _ptr(so), _ptr(sc), _ptr(q)))
        return q

    def unfold_single(self, score=(0, 0, 0, 0)) -> np.ndarray:
        r = int(self.pasur_tree_sizes()[0][0])
        return self.pasur_unfold(np.arange(r + 1, dtype=np.int64), np.tile(np.asarray(score, np.int16), (r, 1)))

    def pasur_cfr_iterate(self, cfg: pasur_config, next_root_util=None):
        nu = None
        if next_root_util is not None:
            nu = next_root_util if hasattr(next_root_util, "data_ptr") else np.ascontiguousarray(next_root_util, np.float32)
        self._c(load().pasur_cfr_iterate(self.h, C.byref(cfg), _ptr(nu)))

    def pasur_cfr_iterate_roots(self, cfg: pasur_config, next_root_util, root_first: int, root_count: int):
        nu = None
        if next_root_util is not None:
            nu = next_root_util if hasattr(next_root_util, "data_ptr") else np.ascontiguousarray(next_root_util, np.float32)
        self._c(load().pasur_cfr_iterate_roots(self.h, C.byref(cfg), _ptr(nu), root_first, root_count))

    def pasur_round_reach(self, root_reach=None, sigma=None) -> np.ndarray:
        """Probability of every next-round root when both follow sigma (default: own sigma-bar)."""
        out = np.zeros(max(self.n_next_roots(), 1), np.float64)
        rr = None if root_reach is None else np.ascontiguousarray(root_reach, np.float64)
        sg = None if sigma is None else (sigma if hasattr(sigma, "data_ptr") else np.ascontiguousarray(sigma, np.float32))
        self._c(load().pasur_round_reach(self.h, _ptr(sg), _ptr(rr), _ptr(out), self.n_next_roots()))
        return out[:self.n_next_roots()]

    def pasur_response_reach(self, mode: int, next_values, root_reach=None, sigma=None) -> np.ndarray:
        """Probability of every next-round root when one player best-responds (mode 1 Alex, 2 Bob;
        3 both on sigma) and the other follows sigma (default: own sigma-bar)."""
        out = np.zeros(max(self.n_next_roots(), 1), np.float64)
        rr = None if root_reach is None else np.ascontiguousarray(root_reach, np.float64)
        sg = None if sigma is None else (sigma if hasattr(sigma, "data_ptr") else np.ascontiguousarray(sigma, np.float32))
        nx = next_values if hasattr(next_values, "data_ptr") else np.ascontiguousarray(next_values, np.float64)
        self._c(load().pasur_response_reach(self.h, mode, _ptr(sg), _ptr(nx), _ptr(rr), _ptr(out), self.n_next_roots()))
        return out[:self.n_next_roots()]

    def pasur_root_sizes(self) -> np.ndarray:
        n = int(self.pasur_tree_sizes()[0][0])
        out = np.zeros(max(n, 1), np.int64)
        self._c(load().pasur_root_sizes(self.h, _ptr(out), n))
        return out[:n]

    def n_edges(self) -> int:
        return int(self.pasur_tree_sizes()[1][1:].sum())

    def pasur_avg_strategy(self, out=None):
        ne = self.n_edges()
        if out is None:
            out = np.zeros(ne, np.float32)
        n = out.numel() if hasattr(out, "numel") else len(out)
        self._c(load().pasur_avg_strategy(self.h, _ptr(out), n))
        return out

    def pasur_avg_strategy_async(self, out):
        """pasur_avg_strategy without waiting: out (host, page-locked for overlap, or device) is
        complete after the context's pasur_sync."""
        n = out.numel() if hasattr(out, "numel") else len(out)
        self._c(load().pasur_avg_strategy_async(self.h, _ptr(out), n))
        return out

    def pasur_round_utilities(self, out=None):
        q0 = int(self.pasur_tree_sizes()[1][0])
        if out is None:
            out = np.zeros(q0, np.float32)
        n = out.numel() if hasattr(out, "numel") else len(out)
        self._c(load().pasur_round_utilities(self.h, _ptr(out), n))
        return out

    def pasur_next_roots(self):
        npool, nroot = C.c_int64(0), C.c_int64(0)
        self._c(load().pasur_next_roots(self.h, None, 0, None, None, 0, None, C.byref(npool), C.byref(nroot)))
        pools = np.zeros(npool.value, np.uint64)
        soff = np.zeros(npool.value + 1, np.int64)
        scores = np.zeros((nroot.value, 4), np.int16)
        lnk = np.zeros(int(self.pasur_tree_sizes()[1][8]), np.int64)
        self._c(load().pasur_next_roots(self.h, _ptr(pools), npool.value, _ptr(soff), _ptr(scores), nroot.value,
                                        _ptr(lnk), C.byref(npool), C.byref(nroot)))
        return pools, soff, scores, lnk

    def pasur_root_values(self, mode: int, sigma=None, next_values=None) -> np.ndarray:
        """fp64 root values: mode 0 minimax, 1 Alex best response, 2 Bob best response, 3 on-policy."""
        q0 = int(self.pasur_tree_sizes()[1][0])
        out = np.zeros(q0, np.float64)
        sg = None if sigma is None else (sigma if hasattr(sigma, "data_ptr") else np.ascontiguousarray(sigma, np.float32))
        nx = None if next_values is None else (next_values if hasattr(next_values, "data_ptr")
                                               else np.ascontiguousarray(next_values, np.float64))
        self._c(load().pasur_root_values(self.h, mode, _ptr(sg), _ptr(nx), _ptr(out), q0))
        return out

    def n_next_roots(self) -> int:
        npool, nroot = C.c_int64(0), C.c_int64(0)
        self._c(load().pasur_next_roots(self.h, None, 0, None, None, 0, None, C.byref(npool), C.byref(nroot)))
        return nroot.value

    def pasur_next_roots_nolinks(self):
        """Next roots without copying the links to the host (they stay on the device)."""
        npool, nroot = C.c_int64(0), C.c_int64(0)
        self._c(load().pasur_next_roots(self.h, None, 0, None, None, 0, None, C.byref(npool), C.byref(nroot)))
        pools = np.zeros(npool.value, np.uint64)
        soff = np.zeros(npool.value + 1, np.int64)
        scores = np.zeros((nroot.value, 4), np.int16)
        self._c(load().pasur_next_roots(self.h, _ptr(pools), npool.value, _ptr(soff), _ptr(scores), nroot.value,
                                        None, C.byref(npool), C.byref(nroot)))
        return pools, soff, scores, None

    def pasur_export_level(self, k: int):
        n = int(self.pasur_tree_sizes()[0][k])
        parent = np.zeros(n, np.int64)
        nchild = np.zeros(n, np.int32)
        lay = np.zeros(n, np.int32)
        pick = np.zeros(n, np.uint64)
        state = np.zeros((n, 3), np.uint64)
        rus = np.zeros((n, 7), np.int8)
        self._c(load().pasur_export_level(self.h, k, n, _ptr(parent), _ptr(nchild), _ptr(lay), _ptr(pick),
                                          _ptr(state), _ptr(rus)))
        return dict(parent=parent, nchild=nchild, lay=lay, pick=pick, state=state, rus=rus)

    def pasur_leaf_values(self, out=None):
        q8 = int(self.pasur_tree_sizes()[1][8])
        if out is None:
            out = np.zeros(q8, np.float32)
        n = out.numel() if hasattr(out, "numel") else len(out)
        self._c(load().pasur_leaf_values(self.h, _ptr(out), n))
        return out

    def pasur_last_cfr_stats(self):
        ms, e, l = C.c_float(0), C.c_int64(0), C.c_int32(0)
        self._c(load().pasur_last_cfr_stats(self.h, C.byref(ms), C.byref(e), C.byref(l)))
        return ms.value, e.value, l.value
