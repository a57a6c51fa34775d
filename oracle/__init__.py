"""FP64 CPU oracle for Force2Vec (arXiv:2009.10035), Python side.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
product library never loads it, and it imports nothing from the product
package.

The arithmetic lives in ``f2v_oracle.c`` (plain C, FP64, optional OpenMP
over the vertices of one minibatch, which Algorithm 2 states as a parallel
loop and which leaves the result bit-identical for any thread count).  This
module compiles it with gcc on first use and marshals numpy arrays into it.

Every function cites the passage it follows:
  philox4x32_10   Philox4x32-10 (Salmon et al., SC'11), the counter-based
                  generator both sides implement from its published definition
  init_embedding  Sec. III-C "Initialization": random Z, uniform [-0.5, 0.5)
  samples         negative samples, s per vertex (Sec. III-C complexity text)
  samples_shared  Alg. 1's sampling step read literally: one S_b per minibatch
  partition       Alg. 1's partition step read literally: new each epoch
  grad_minibatch  Algorithm 2, per-pair terms Eq. 5/6 (sigmoid), Eq. 8/9 (t),
                  Table "diffmodels" (FR, LinLog, ForceAtlas)
  walk            Algorithm 3 (GenWalk), the rForce2Vec neighbourhood
  train           Algorithm 1 with the SGD update of Eq. 10 (walk > 0:
                  rForce2Vec, N(u) from Algorithm 3)
  loss_vertex     Eq. 2 with Eq. 3 (sigmoid) or Eq. 7 (t)
  scores, auc     held-out-edge link prediction, Mann-Whitney AUC
  downstream      (submodule, numpy) Sec. IV's link prediction with Hadamard
                  features and logistic regression, k-means and modularity
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

TDIST = 0
SIGMOID = 1
FR = 2            # Fruchterman-Reingold (Table "diffmodels")
LINLOG = 3
FORCEATLAS = 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "f2v_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libf2v_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libf2v_oracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # -ffp-contract=off: no fused multiply-add, so each FP64 operation rounds
    # exactly as written.
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32, i64, u32, u64, f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
        vp = ctypes.c_void_p
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
        lib.orc_philox4x32_10.restype = None
        lib.orc_init_value.argtypes = [u64, u32, u32]
        lib.orc_init_value.restype = f64
        lib.orc_init_embedding.argtypes = [i64, i32, u64, vp]
        lib.orc_init_embedding.restype = None
        lib.orc_sample.argtypes = [u64, u32, u32, u32, u32]
        lib.orc_sample.restype = u32
        lib.orc_samples.argtypes = [u64, i64, i32, i32, vp]
        lib.orc_samples.restype = None
        lib.orc_grad_minibatch.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, i64, i64,
                                           i32, u64, i32, vp, vp, vp]
        lib.orc_grad_minibatch.restype = None
        lib.orc_grad_minibatch_abs.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, vp, i64,
                                               i64, i32, u64, i32, vp, vp, vp, vp]
        lib.orc_grad_minibatch_abs.restype = None
        lib.orc_grad_minibatch_ex.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, vp, i64, i64,
                                              i32, i32, i64, u64, i32, vp, vp, vp, vp]
        lib.orc_grad_minibatch_ex.restype = None
        lib.orc_sample_shared.argtypes = [u64, u32, u32, u32, u32]
        lib.orc_sample_shared.restype = u32
        lib.orc_walk.argtypes = [u64, vp, vp, i64, i32, i32, vp]
        lib.orc_walk.restype = None
        lib.orc_train_ex.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, i32, i32, i32, i32,
                                     i64, u64, f64, i32, i32, i32, i32, i64, vp, vp]
        lib.orc_grad_core.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, vp, vp, i64, i64, i32,
                                      i32, i64, i64, u64, i32, vp, vp, vp, vp]
        lib.orc_grad_core.restype = None
        lib.orc_partition.argtypes = [u64, i64, i32, vp]
        lib.orc_partition.restype = ctypes.c_int
        lib.orc_train_ex.restype = ctypes.c_int
        lib.orc_learning_rate.argtypes = [f64, i32, i32, i32]
        lib.orc_learning_rate.restype = f64
        lib.orc_train.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, i32, i64, u64,
                                  f64, i32, i32, i32, i32, i64, vp, vp]
        lib.orc_train.restype = ctypes.c_int
        lib.orc_loss_vertex.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, i64, i32, u64,
                                        i32, vp, vp]
        lib.orc_loss_vertex.restype = f64
        lib.orc_loss_total.argtypes = [ctypes.c_int, i64, i32, vp, vp, vp, i32, u64, i32,
                                       vp, vp]
        lib.orc_loss_total.restype = f64
        lib.orc_scores.argtypes = [ctypes.c_int, i32, vp, vp, i64, vp]
        lib.orc_scores.restype = None
        lib.orc_auc.argtypes = [vp, i64, vp, i64]
        lib.orc_auc.restype = f64
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    """Sets the oracle's OpenMP thread count (n <= 0 keeps it); returns it."""
    return int(_load().orc_set_threads(int(n)))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(row_ptr, col_idx):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    if col_idx.size == 0:
        col_idx = np.zeros(1, dtype=np.int32)   # a valid pointer for an empty graph
    return row_ptr, col_idx


def _injected(samples):
    """samples: None (Philox) or a list of per-vertex index lists S(u)."""
    if samples is None:
        return None, None
    ptr = np.zeros(len(samples) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(x) for x in samples])
    idx = np.zeros(max(int(ptr[-1]), 1), dtype=np.int32)
    if ptr[-1]:
        idx[:ptr[-1]] = np.concatenate([np.asarray(x, dtype=np.int32) for x in samples if len(x)])
    return ptr, idx


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def init_embedding(n: int, d: int, seed: int) -> np.ndarray:
    """Z0 (n x d, FP64), uniform in [-0.5, 0.5) from Philox."""
    lib = _load()
    Z = np.zeros((n, d), dtype=np.float64)
    lib.orc_init_embedding(n, d, seed, _ptr(Z))
    return Z


def samples(n: int, s: int, epoch: int, seed: int) -> np.ndarray:
    """Negative-sample indices of one epoch, an n x s int32 array."""
    lib = _load()
    out = np.zeros((n, s), dtype=np.int32)
    if n and s:
        lib.orc_samples(seed, n, s, epoch, _ptr(out))
    return out


def walk(row_ptr, col_idx, u: int, epoch: int, k: int, seed: int) -> np.ndarray:
    """Algorithm 3 for vertex u in epoch `epoch`: the k vertices the walk
    reaches, -1 once it has stopped at a vertex without neighbours."""
    lib = _load()
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    out = np.zeros(max(k, 1), dtype=np.int32)
    if k > 0:
        lib.orc_walk(seed, _ptr(row_ptr), _ptr(col_idx), u, epoch, k, _ptr(out))
    return out[:k]


def samples_shared(n: int, s: int, b: int, epoch: int, seed: int) -> np.ndarray:
    """Algorithm 1's sampling step read literally: row u lists the set S_b of u's
    minibatch (k = u // b), an n x s int32 array."""
    lib = _load()
    out = np.zeros((n, s), dtype=np.int32)
    for u in range(0, n, b):
        row = [lib.orc_sample_shared(seed, u // b, epoch, j, n) for j in range(s)]
        out[u:min(n, u + b)] = row
    return out


def grad_minibatch(model, row_ptr, col_idx, Z, u_begin, u_end, s, seed, epoch,
                   injected=None, walk=0, shared_b=0) -> np.ndarray:
    """Algorithm 2 for the vertices [u_begin, u_end); returns (u_end-u_begin) x d.
    walk > 0: N(u) from Algorithm 3 (rForce2Vec).  shared_b > 0: every
    vertex of minibatch k = u // shared_b uses that minibatch's sample set."""
    return grad_minibatch_abs(model, row_ptr, col_idx, Z, u_begin, u_end, s, seed, epoch,
                              injected=injected, walk=walk, shared_b=shared_b)[0]


def grad_minibatch_abs(model, row_ptr, col_idx, Z, u_begin, u_end, s, seed, epoch,
                       injected=None, gather=None, walk=0, shared_b=0):
    """Algorithm 2 for [u_begin, u_end): returns (grad, grad_abs), where
    grad_abs sums the absolute values of the per-pair terms element by
    element (the scale of the rounding error of an FP32 evaluation).  With
    `gather`, partner rows come from that matrix and only z_u from Z.
    walk > 0: N(u) from Algorithm 3 (rForce2Vec).  shared_b > 0: shared
    sample sets of minibatches of that size."""
    lib = _load()
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    n, d = Z.shape
    Zp = None if gather is None else np.ascontiguousarray(gather, dtype=np.float64)
    assert Zp is None or Zp.shape == Z.shape
    sp, si = _injected(injected)
    g = np.zeros((u_end - u_begin, d), dtype=np.float64)
    ga = np.zeros((u_end - u_begin, d), dtype=np.float64)
    lib.orc_grad_minibatch_ex(model, n, d, _ptr(row_ptr), _ptr(col_idx), _ptr(Z),
                              None if Zp is None else _ptr(Zp), u_begin, u_end, s, int(walk),
                              int(shared_b), seed, epoch, _ptr(sp), _ptr(si), _ptr(g), _ptr(ga))
    return g, ga


def partition(n: int, epoch: int, seed: int) -> np.ndarray:
    """The random partition of an epoch (the partition step of Alg. 1): the vertices in
    minibatch order; minibatch k is positions [k b, (k+1) b)."""
    lib = _load()
    perm = np.zeros(max(n, 1), dtype=np.int64)
    if lib.orc_partition(seed, n, epoch, _ptr(perm)) != 0:
        raise MemoryError("oracle partition: out of memory")
    return perm[:n]


def grad_vertices_abs(model, row_ptr, col_idx, Z, verts, s, seed, epoch, gather=None, walk=0,
                      shared_k=-1):
    """Algorithm 2 for the vertex list `verts` (one minibatch of a random
    partition): returns (grad, grad_abs), rows in list order.  shared_k >= 0:
    the shared sample set of minibatch shared_k."""
    lib = _load()
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    n, d = Z.shape
    Zp = None if gather is None else np.ascontiguousarray(gather, dtype=np.float64)
    v = np.ascontiguousarray(verts, dtype=np.int64)
    g = np.zeros((v.size, d), dtype=np.float64)
    ga = np.zeros((v.size, d), dtype=np.float64)
    if v.size:
        lib.orc_grad_core(model, n, d, _ptr(row_ptr), _ptr(col_idx), _ptr(Z),
                          None if Zp is None else _ptr(Zp), _ptr(v), 0, v.size, s, int(walk),
                          int(shared_k), 0, seed, epoch, None, None, _ptr(g), _ptr(ga))
    return g, ga


def learning_rate(lr0: float, schedule: int, total_epochs: int, epoch: int) -> float:
    return _load().orc_learning_rate(lr0, schedule, total_epochs, epoch)


def train(model, row_ptr, col_idx, Z, s, b, seed, lr, epochs, start_epoch=0,
          schedule=0, total_epochs=0, max_minibatches=-1, injected=None,
          walk=0, shared=False, partition=False) -> np.ndarray:
    """Algorithm 1 from embedding Z (copied); returns the new FP64 embedding.
    walk > 0: rForce2Vec, N(u) from Algorithm 3 with walks of that length.
    shared: one sample set S_b per minibatch (the sampling step read literally).
    partition: a new random partition every epoch (the partition step read literally)."""
    lib = _load()
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    Z = np.array(Z, dtype=np.float64, order="C", copy=True)
    n, d = Z.shape
    sp, si = _injected(injected)
    rc = lib.orc_train_ex(model, n, d, _ptr(row_ptr), _ptr(col_idx), _ptr(Z), s, int(walk),
                          int(bool(shared)), int(bool(partition)), b, seed, lr, schedule,
                          total_epochs, start_epoch, epochs, max_minibatches, _ptr(sp),
                          _ptr(si))
    if rc != 0:
        raise MemoryError("oracle train: out of memory")
    return Z


def loss_vertex(model, row_ptr, col_idx, Z, u, s, seed, epoch, injected=None) -> float:
    lib = _load()
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    n, d = Z.shape
    sp, si = _injected(injected)
    return lib.orc_loss_vertex(model, n, d, _ptr(row_ptr), _ptr(col_idx), _ptr(Z), u, s,
                               seed, epoch, _ptr(sp), _ptr(si))


def loss_total(model, row_ptr, col_idx, Z, s, seed, epoch, injected=None) -> float:
    lib = _load()
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    n, d = Z.shape
    sp, si = _injected(injected)
    return lib.orc_loss_total(model, n, d, _ptr(row_ptr), _ptr(col_idx), _ptr(Z), s, seed,
                              epoch, _ptr(sp), _ptr(si))


def scores(model, Z, pairs) -> np.ndarray:
    lib = _load()
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(pairs.shape[0], dtype=np.float64)
    if pairs.shape[0]:
        lib.orc_scores(model, Z.shape[1], _ptr(Z), _ptr(pairs), pairs.shape[0], _ptr(out))
    return out


def auc(pos_scores, neg_scores) -> float:
    lib = _load()
    pos = np.ascontiguousarray(pos_scores, dtype=np.float64)
    neg = np.array(neg_scores, dtype=np.float64, copy=True)
    return lib.orc_auc(_ptr(pos), pos.size, _ptr(neg), neg.size)


def link_auc(model, Z, pos_pairs, neg_pairs) -> float:
    """Held-out-edge AUC of embedding Z (FP64)."""
    return auc(scores(model, Z, pos_pairs), scores(model, Z, neg_pairs))
