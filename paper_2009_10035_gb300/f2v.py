"""Python binding of libf2v (the C ABI in include/f2v.h).

Argument marshalling only: every step of an epoch runs in the library's CUDA
kernels.  If the library has not been built this module raises on first use;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

TDIST = 0
SIGMOID = 1
FR = 2              # Fruchterman-Reingold
LINLOG = 3
FORCEATLAS = 4
FP32 = 0
BF16 = 1
LR_CONSTANT = 0
LR_LINEAR = 1
FLAG_CHECK_SYMMETRY = 0x1
FLAG_NO_STAGING = 0x2
FLAG_SHARED_SAMPLES = 0x4
FLAG_RANDOM_PARTITION = 0x8

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = range(6)
_STATUS = {0: "F2V_OK", 1: "F2V_EINVAL", 2: "F2V_ENOMEM", 3: "F2V_ECUDA",
           4: "F2V_ETIMEOUT", 5: "F2V_ESTATE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libf2v.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
HEADER = os.path.join(INCLUDE, "f2v.h")

_lock = threading.Lock()
_lib = None


class F2VError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def header_functions() -> list[str]:
    """Names of the functions the headers under include/ declare."""
    names = set()
    for fn in sorted(os.listdir(INCLUDE)):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(INCLUDE, fn)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(f2v_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def signatures() -> dict:
    """ctypes (argument types, result type) of every function of the C ABI."""
    i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    vp, sz, f32, st = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_float, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    return {
        "f2v_create": ([vp, vp, i32, i32, st, i32, f32, i32, u64, pp], st),
        "f2v_create_ex": ([vp, vp, i32, i32, st, i32, f32, i32, u64, st, u32, vp, pp], st),
        "f2v_create_rw": ([vp, vp, i32, i32, st, i32, i32, f32, i32, u64, st, u32, vp, pp],
                          st),
        "f2v_destroy": ([vp], None),
        "f2v_epoch": ([vp], st),
        "f2v_train": ([vp, i32], st),
        "f2v_run_minibatches": ([vp, i32], st),
        "f2v_get_progress": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32)], st),
        "f2v_synchronize": ([vp], st),
        "f2v_get_embedding": ([vp, vp, sz], st),
        "f2v_get_embedding_device": ([vp, vp, sz], st),
        "f2v_set_embedding": ([vp, vp, sz], st),
        "f2v_set_lr": ([vp, f32], st),
        "f2v_set_schedule": ([vp, st, i32], st),
        "f2v_set_epoch": ([vp, i32], st),
        "f2v_get_epoch": ([vp, ctypes.POINTER(i32)], st),
        "f2v_set_stream": ([vp, vp], st),
        "f2v_eval_auc": ([vp, vp, i64, vp, i64, ctypes.POINTER(ctypes.c_double)], st),
        "f2v_eval_loss": ([vp, i32, ctypes.POINTER(ctypes.c_double)], st),
        "f2v_debug_samples": ([vp, i32, vp, sz], st),
        "f2v_debug_walks": ([vp, i32, vp, sz], st),
        "f2v_debug_wait": ([vp, i32], st),
        "f2v_eval_link_lr": ([vp, vp, i64, vp, i64, vp, ctypes.POINTER(ctypes.c_double),
                              vp], st),
        "f2v_eval_kmeans": ([vp, i32, vp, i32, vp, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(i32)], st),
        "f2v_pairs_per_epoch": ([vp, ctypes.POINTER(i64)], st),
        "f2v_device_bytes": ([vp, ctypes.POINTER(sz)], st),
        "f2v_launch_count": ([vp, ctypes.POINTER(i64)], st),
        "f2v_set_kernel_timing": ([vp, i32], st),
        "f2v_read_kernel_timing": ([vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)], st),
        "f2v_minibatch_noalloc": ([vp, vp, i32, i32, st, i32, f32, u64, i32, i32, i32, vp,
                                   vp, vp], st),
        "f2v_noalloc_last_error": ([], ctypes.c_char_p),
        "f2v_last_error": ([vp], ctypes.c_char_p),
        "f2v_last_error_global": ([], ctypes.c_char_p),
        # batched form (include/f2v_batch.h)
        "f2v_batch_create": ([i32, vp, vp, vp, vp, vp, st, i32, f32, i32, st, vp, pp], st),
        "f2v_batch_destroy": ([vp], None),
        "f2v_batch_epoch": ([vp], st),
        "f2v_batch_train": ([vp, i32], st),
        "f2v_batch_synchronize": ([vp], st),
        "f2v_batch_run_minibatches": ([vp, i32], st),
        "f2v_batch_get_progress": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i32)], st),
        "f2v_batch_set_lr": ([vp, f32], st),
        "f2v_batch_set_schedule": ([vp, st, i32], st),
        "f2v_batch_get_epoch": ([vp, ctypes.POINTER(i32)], st),
        "f2v_batch_get_embedding": ([vp, i32, vp, sz], st),
        "f2v_batch_get_embeddings": ([vp, vp, sz], st),
        "f2v_batch_set_embedding": ([vp, i32, vp, sz], st),
        "f2v_batch_set_tiling": ([vp, vp], st),
        "f2v_batch_get_tiling": ([vp, i32, vp], st),
        "f2v_batch_autotune": ([vp, i32, vp, i32, ctypes.POINTER(i32)], st),
        "f2v_batch_pairs_per_epoch": ([vp, ctypes.POINTER(i64)], st),
        "f2v_batch_bytes_per_epoch": ([vp, ctypes.POINTER(i64)], st),
        "f2v_batch_device_bytes": ([vp, ctypes.POINTER(sz)], st),
        "f2v_batch_num_graphs": ([vp, ctypes.POINTER(i32)], st),
        "f2v_batch_launch_count": ([vp, ctypes.POINTER(i64)], st),
        "f2v_batch_stream": ([vp, pp], st),
        "f2v_batch_last_error": ([vp], ctypes.c_char_p),
        # served form (include/f2v_serve.h)
        "f2v_server_create": ([sz, i32, pp], st),
        "f2v_server_submit": ([vp, vp, ctypes.POINTER(i64)], st),
        "f2v_server_job": ([vp, i64, vp], st),
        "f2v_server_wait": ([vp, i64], st),
        "f2v_server_wait_all": ([vp], st),
        "f2v_server_get_stats": ([vp, vp], st),
        "f2v_server_destroy": ([vp], None),
        "f2v_server_last_error": ([vp], ctypes.c_char_p),
        "f2v_server_job_error": ([vp, i64], ctypes.c_char_p),
    }


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Loads libf2v.so and declares its signatures (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libf2v.so is not built ({p}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(p)
        for name, (args, res) in signatures().items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        if path is None:
            _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _host_out(out, count: int, exact: bool = True) -> np.ndarray:
    """Checks a caller's output buffer: writable, C-contiguous float32 with
    `count` elements (at least `count` where exact is False)."""
    if not isinstance(out, np.ndarray) or out.dtype != np.float32:
        raise ValueError("output must be a float32 numpy array")
    if not out.flags.c_contiguous or not out.flags.writeable:
        raise ValueError("output must be C-contiguous and writable")
    if (out.size != count) if exact else (out.size < count):
        raise ValueError(f"output holds {out.size} floats, needs {count}")
    return out


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)       # a torch.cuda.Stream


class Context:
    """One embedding job: a graph, its device-resident Z and the epoch counter.
    walk_length > 0 makes it rForce2Vec (f2v_create_rw): N(u) from random
    walks of that many steps (Algorithm 3) instead of u's neighbours."""

    def __init__(self, row_ptr, col_idx, n: int, d: int, model: int = TDIST, s: int = 5,
                 lr: float = 0.02, minibatch: int = 256, seed: int = 1,
                 precision: int = FP32, flags: int = 0, stream=None, walk_length: int = 0):
        self._lib = load_library()
        self.n, self.d, self.s = int(n), int(d), int(s)
        self.walk_length = int(walk_length)
        self.model, self.precision = int(model), int(precision)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        if rp.size != self.n + 1:
            raise ValueError(f"row_ptr has {rp.size} entries, expected n+1 = {self.n + 1}")
        if ci.size == 0:
            ci = np.zeros(1, dtype=np.int32)
        h = ctypes.c_void_p()
        if self.walk_length:
            rc = self._lib.f2v_create_rw(_ptr(rp), _ptr(ci), self.n, self.d, int(model), self.s,
                                         self.walk_length, float(lr), int(minibatch),
                                         int(seed) & (2**64 - 1), int(precision), int(flags),
                                         _stream_handle(stream), ctypes.byref(h))
        else:
            rc = self._lib.f2v_create_ex(_ptr(rp), _ptr(ci), self.n, self.d, int(model), self.s,
                                         float(lr), int(minibatch), int(seed) & (2**64 - 1),
                                         int(precision), int(flags), _stream_handle(stream),
                                         ctypes.byref(h))
        if rc != OK:
            raise F2VError(rc, self._lib.f2v_last_error_global().decode())
        self._h = h

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc: int):
        if rc != OK:
            msg = self._lib.f2v_last_error(self._h).decode() if self._h else ""
            raise F2VError(rc, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.f2v_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Algorithm 1 ------------------------------------------------------
    def epoch(self):
        self._check(self._lib.f2v_epoch(self._h))

    def train(self, epochs: int):
        self._check(self._lib.f2v_train(self._h, int(epochs)))

    def run_minibatches(self, count: int):
        self._check(self._lib.f2v_run_minibatches(self._h, int(count)))

    @property
    def progress(self) -> tuple[int, int]:
        e = ctypes.c_int32()
        k = ctypes.c_int32()
        self._check(self._lib.f2v_get_progress(self._h, ctypes.byref(e), ctypes.byref(k)))
        return e.value, k.value

    def synchronize(self):
        self._check(self._lib.f2v_synchronize(self._h))

    def embedding(self) -> np.ndarray:
        out = np.empty((self.n, self.d), dtype=np.float32)
        self._check(self._lib.f2v_get_embedding(self._h, _ptr(out), out.size))
        return out

    def embedding_into_host(self, out: np.ndarray):
        _host_out(out, self.n * self.d)
        self._check(self._lib.f2v_get_embedding(self._h, _ptr(out), out.size))

    def embedding_into_device(self, dev_ptr: int):
        self._check(self._lib.f2v_get_embedding_device(self._h, ctypes.c_void_p(dev_ptr),
                                                       self.n * self.d))

    def set_embedding(self, z):
        z = np.ascontiguousarray(z, dtype=np.float32)
        self._check(self._lib.f2v_set_embedding(self._h, _ptr(z), z.size))

    def set_lr(self, lr: float):
        self._check(self._lib.f2v_set_lr(self._h, float(lr)))

    def set_schedule(self, schedule: int, total_epochs: int):
        self._check(self._lib.f2v_set_schedule(self._h, int(schedule), int(total_epochs)))

    def set_epoch(self, epoch: int):
        self._check(self._lib.f2v_set_epoch(self._h, int(epoch)))

    @property
    def epoch_counter(self) -> int:
        e = ctypes.c_int32()
        self._check(self._lib.f2v_get_epoch(self._h, ctypes.byref(e)))
        return e.value

    def set_stream(self, stream):
        self._check(self._lib.f2v_set_stream(self._h, _stream_handle(stream)))

    # -- evaluation and introspection -------------------------------------
    def eval_auc(self, pos_pairs, neg_pairs) -> float:
        pos = np.ascontiguousarray(pos_pairs, dtype=np.int32).reshape(-1, 2)
        neg = np.ascontiguousarray(neg_pairs, dtype=np.int32).reshape(-1, 2)
        out = ctypes.c_double()
        self._check(self._lib.f2v_eval_auc(self._h, _ptr(pos), pos.shape[0], _ptr(neg),
                                           neg.shape[0], ctypes.byref(out)))
        return out.value

    def eval_loss(self, epoch: int) -> float:
        """The loss of Eq. 2 (Eq. 3 / Eq. 7) on the current Z in FP64, with
        the negative samples of `epoch`."""
        out = ctypes.c_double()
        self._check(self._lib.f2v_eval_loss(self._h, int(epoch), ctypes.byref(out)))
        return out.value

    def debug_samples(self, epoch: int) -> np.ndarray:
        out = np.zeros((self.n, self.s), dtype=np.int32)
        buf = out if out.size else np.zeros(1, np.int32)
        self._check(self._lib.f2v_debug_samples(self._h, int(epoch), _ptr(buf), out.size))
        return out

    def eval_link_lr(self, pos_pairs, neg_pairs, train_mask):
        """Sec. IV link prediction: Hadamard features, logistic regression
        fitted on train_mask (pos pairs first), accuracy on the rest.
        Returns (accuracy, theta = (w, b))."""
        pos = np.ascontiguousarray(pos_pairs, dtype=np.int32).reshape(-1, 2)
        neg = np.ascontiguousarray(neg_pairs, dtype=np.int32).reshape(-1, 2)
        mask = np.ascontiguousarray(train_mask, dtype=np.uint8)
        if mask.size != pos.shape[0] + neg.shape[0]:
            raise ValueError("train_mask must have one entry per pair")
        acc = ctypes.c_double()
        theta = np.zeros(self.d + 1, dtype=np.float64)
        self._check(self._lib.f2v_eval_link_lr(self._h, _ptr(pos), pos.shape[0], _ptr(neg),
                                               neg.shape[0], _ptr(mask), ctypes.byref(acc),
                                               _ptr(theta)))
        return acc.value, theta

    def eval_kmeans(self, init, iters: int = 100):
        """Sec. IV clustering: k-means from centres Z[init]; returns
        (modularity, labels, rounds)."""
        init = np.ascontiguousarray(init, dtype=np.int32)
        labels = np.zeros(self.n, dtype=np.int32)
        q = ctypes.c_double()
        r = ctypes.c_int32()
        self._check(self._lib.f2v_eval_kmeans(self._h, init.size, _ptr(init), int(iters),
                                              _ptr(labels), ctypes.byref(q), ctypes.byref(r)))
        return q.value, labels, r.value

    def debug_wait(self, kind: int):
        """Runs the bounded-wait test of f2v_debug_wait (raises F2VError
        with F2V_ETIMEOUT for kinds 1-3)."""
        self._check(self._lib.f2v_debug_wait(self._h, int(kind)))

    def debug_walks(self, epoch: int) -> np.ndarray:
        """n x walk_length: the vertex each walk step reaches, -1 where the
        step exerts no force."""
        out = np.zeros((self.n, self.walk_length), dtype=np.int32)
        buf = out if out.size else np.zeros(1, np.int32)
        self._check(self._lib.f2v_debug_walks(self._h, int(epoch), _ptr(buf), out.size))
        return out

    @property
    def pairs_per_epoch(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.f2v_pairs_per_epoch(self._h, ctypes.byref(v)))
        return v.value

    @property
    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        self._check(self._lib.f2v_device_bytes(self._h, ctypes.byref(v)))
        return v.value

    @property
    def launch_count(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.f2v_launch_count(self._h, ctypes.byref(v)))
        return v.value

    def set_kernel_timing(self, enable: bool):
        self._check(self._lib.f2v_set_kernel_timing(self._h, 1 if enable else 0))

    def read_kernel_timing(self) -> tuple[int, float]:
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        self._check(self._lib.f2v_read_kernel_timing(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value


def create(graph, d: int, **kw) -> Context:
    """Context for a ``graphs.Graph``."""
    return Context(graph.row_ptr, graph.col_idx, graph.n, d, **kw)


class Tiling(ctypes.Structure):
    """f2v_tiling: lanes per row (L) and pairs per item (C) for row size d."""
    _fields_ = [("d", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32),
                ("item_pairs", ctypes.c_int32)]

    def as_tuple(self) -> tuple[int, int, int]:
        return (self.d, self.lanes_per_row, self.item_pairs)


class Batch:
    """Many graphs trained together (include/f2v_batch.h): one persistent
    kernel launch per row shape and epoch, replayed from a CUDA graph."""

    def __init__(self, n, d, seed, row_ptr, col_idx, model: int = TDIST, s: int = 5,
                 lr: float = 0.02, minibatch: int = 128, precision: int = FP32, stream=None):
        self._lib = load_library()
        self.n = np.ascontiguousarray(n, np.int32)
        self.d = np.ascontiguousarray(d, np.int32)
        sd = np.ascontiguousarray(np.asarray(seed).astype(np.uint64))
        rp = np.ascontiguousarray(row_ptr, np.int32)
        ci = np.ascontiguousarray(col_idx, np.int32)
        if ci.size == 0:
            ci = np.zeros(1, np.int32)
        G = int(self.n.size)
        if self.d.size != G or sd.size != G:
            raise ValueError("n, d and seed must have one entry per graph")
        if rp.size != int(self.n.astype(np.int64).sum()) + G:
            raise ValueError("row_ptr must hold n[g] + 1 entries per graph")
        self.s, self.model, self.precision = int(s), int(model), int(precision)
        h = ctypes.c_void_p()
        rc = self._lib.f2v_batch_create(G, _ptr(self.n), _ptr(self.d), _ptr(sd), _ptr(rp),
                                        _ptr(ci), int(model), int(s), float(lr), int(minibatch),
                                        int(precision), _stream_handle(stream), ctypes.byref(h))
        if rc != OK:
            raise F2VError(rc, self._lib.f2v_last_error_global().decode())
        self._h = h
        self.z_off = np.zeros(G + 1, np.int64)
        self.z_off[1:] = np.cumsum(self.n.astype(np.int64) * self.d)

    @classmethod
    def from_graphs(cls, batch, **kw) -> "Batch":
        """Batch over a ``graphs.GraphBatch`` (its n, d, seeds and CSRs)."""
        return cls(batch.n, batch.d, batch.seed, batch.row_ptr, batch.col_idx, **kw)

    def _check(self, rc: int):
        if rc != OK:
            msg = self._lib.f2v_batch_last_error(self._h).decode() if self._h else ""
            raise F2VError(rc, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.f2v_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_graphs(self) -> int:
        return int(self.n.size)

    def epoch(self):
        self._check(self._lib.f2v_batch_epoch(self._h))

    def train(self, epochs: int):
        self._check(self._lib.f2v_batch_train(self._h, int(epochs)))

    def run_minibatches(self, count: int):
        self._check(self._lib.f2v_batch_run_minibatches(self._h, int(count)))

    @property
    def progress(self) -> tuple[int, int]:
        e = ctypes.c_int32()
        k = ctypes.c_int32()
        self._check(self._lib.f2v_batch_get_progress(self._h, ctypes.byref(e), ctypes.byref(k)))
        return e.value, k.value

    def synchronize(self):
        self._check(self._lib.f2v_batch_synchronize(self._h))

    def set_lr(self, lr: float):
        self._check(self._lib.f2v_batch_set_lr(self._h, float(lr)))

    def set_schedule(self, schedule: int, total_epochs: int):
        self._check(self._lib.f2v_batch_set_schedule(self._h, int(schedule), int(total_epochs)))

    @property
    def epoch_counter(self) -> int:
        e = ctypes.c_int32()
        self._check(self._lib.f2v_batch_get_epoch(self._h, ctypes.byref(e)))
        return e.value

    def embedding(self, g: int) -> np.ndarray:
        out = np.empty((int(self.n[g]), int(self.d[g])), np.float32)
        self._check(self._lib.f2v_batch_get_embedding(self._h, int(g), _ptr(out), out.size))
        return out

    def embeddings_into_host(self, out: np.ndarray):
        """All graphs' Z, concatenated in graph order (row-major per graph)."""
        _host_out(out, int(self.z_off[-1]))
        self._check(self._lib.f2v_batch_get_embeddings(self._h, _ptr(out), out.size))

    def set_embedding(self, g: int, z):
        z = np.ascontiguousarray(z, np.float32)
        self._check(self._lib.f2v_batch_set_embedding(self._h, int(g), _ptr(z), z.size))

    def set_tiling(self, d: int, lanes_per_row: int, item_pairs: int):
        t = Tiling(int(d), int(lanes_per_row), int(item_pairs))
        self._check(self._lib.f2v_batch_set_tiling(self._h, ctypes.byref(t)))

    def tiling(self, d: int) -> tuple[int, int, int]:
        t = Tiling()
        self._check(self._lib.f2v_batch_get_tiling(self._h, int(d), ctypes.byref(t)))
        return t.as_tuple()

    def autotune(self, epochs_per_candidate: int = 1, cache: str | None = None,
                 key: str | None = None) -> list[tuple[int, int, int]]:
        """Times candidate tilings on this batch and applies the fastest
        (embeddings and epoch counter are restored).  With `cache` (a JSON
        file) and `key`, a tiling found earlier under `key` is applied
        instead, and a new one is stored there."""
        import json
        if cache and key and os.path.exists(cache):
            with open(cache) as f:
                known = json.load(f)
            if key in known:
                for d, L, C in known[key]:
                    self.set_tiling(d, L, C)
                return [tuple(x) for x in known[key]]
        arr = (Tiling * 8)()
        cnt = ctypes.c_int32()
        self._check(self._lib.f2v_batch_autotune(self._h, int(epochs_per_candidate), arr, 8,
                                                 ctypes.byref(cnt)))
        chosen = [arr[i].as_tuple() for i in range(cnt.value)]
        if cache and key:
            known = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f)
            known[key] = [list(t) for t in chosen]
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(known, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return chosen

    @property
    def pairs_per_epoch(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.f2v_batch_pairs_per_epoch(self._h, ctypes.byref(v)))
        return v.value

    @property
    def bytes_per_epoch(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.f2v_batch_bytes_per_epoch(self._h, ctypes.byref(v)))
        return v.value

    @property
    def device_bytes(self) -> int:
        v = ctypes.c_size_t()
        self._check(self._lib.f2v_batch_device_bytes(self._h, ctypes.byref(v)))
        return v.value

    @property
    def launch_count(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.f2v_batch_launch_count(self._h, ctypes.byref(v)))
        return v.value

    @property
    def stream(self) -> int:
        v = ctypes.c_void_p()
        self._check(self._lib.f2v_batch_stream(self._h, ctypes.byref(v)))
        return v.value or 0


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = range(4)


class JobSpec(ctypes.Structure):
    """f2v_job."""
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("n", ctypes.c_int32), ("d", ctypes.c_int32), ("model", ctypes.c_int),
                ("s", ctypes.c_int32), ("lr", ctypes.c_float), ("minibatch", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("epochs", ctypes.c_int32),
                ("precision", ctypes.c_int), ("out", ctypes.c_void_p)]


class JobInfo(ctypes.Structure):
    """f2v_job_info."""
    _fields_ = [("state", ctypes.c_int32), ("epochs_done", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("finish_s", ctypes.c_double), ("pairs", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("status", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    """f2v_server_stats."""
    _fields_ = [("submitted", ctypes.c_int64), ("done", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("running", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("pairs_done", ctypes.c_int64), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("budget", ctypes.c_size_t),
                ("busy_s", ctypes.c_double)]


class Server:
    """Job server with continuous batching (include/f2v_serve.h).  The arrays
    of a submitted job are kept alive here until the job is collected."""

    def __init__(self, budget_bytes: int, max_active: int = 1 << 20):
        self._lib = load_library()
        h = ctypes.c_void_p()
        rc = self._lib.f2v_server_create(int(budget_bytes), int(max_active), ctypes.byref(h))
        if rc != OK:
            raise F2VError(rc, self._lib.f2v_last_error_global().decode())
        self._h = h
        self._keep = {}

    def _check(self, rc: int):
        if rc != OK:
            raise F2VError(rc, self._lib.f2v_server_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.f2v_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, row_ptr, col_idx, n: int, d: int, model: int = TDIST, s: int = 5,
               lr: float = 0.02, minibatch: int = 4096, seed: int = 1, epochs: int = 10,
               precision: int = FP32, out: np.ndarray | None = None) -> int:
        """Enqueues a job; returns its id.  `out` (n x d float32, C order)
        receives Z when the job completes (allocated here if not given)."""
        rp = np.ascontiguousarray(row_ptr, np.int32)
        ci = np.ascontiguousarray(col_idx, np.int32)
        if ci.size == 0:
            ci = np.zeros(1, np.int32)
        if out is None:
            out = np.empty((int(n), int(d)), np.float32)
        _host_out(out, int(n) * int(d), exact=False)
        spec = JobSpec(_ptr(rp).value, _ptr(ci).value, int(n), int(d), int(model), int(s),
                       float(lr), int(minibatch), int(seed) & (2**64 - 1), int(epochs),
                       int(precision), _ptr(out).value)
        jid = ctypes.c_int64()
        self._check(self._lib.f2v_server_submit(self._h, ctypes.byref(spec), ctypes.byref(jid)))
        self._keep[jid.value] = (rp, ci, out)
        return jid.value

    def info(self, jid: int) -> JobInfo:
        info = JobInfo()
        self._check(self._lib.f2v_server_job(self._h, int(jid), ctypes.byref(info)))
        return info

    def wait(self, jid: int) -> np.ndarray:
        """Waits for job `jid` and returns its Z (raises if it failed)."""
        rc = self._lib.f2v_server_wait(self._h, int(jid))
        if rc != OK:
            raise F2VError(rc, self._lib.f2v_server_job_error(self._h, int(jid)).decode())
        rp, ci, out = self._keep.pop(int(jid))
        return out

    def wait_all(self):
        self._lib.f2v_server_wait_all(self._h)

    def forget(self, jid: int):
        """Drops the references kept for a finished job."""
        self._keep.pop(int(jid), None)

    def stats(self) -> ServerStats:
        st = ServerStats()
        self._check(self._lib.f2v_server_get_stats(self._h, ctypes.byref(st)))
        return st
