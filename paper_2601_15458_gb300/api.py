"""Python entry points over the C ABI of ``include/msa.h``.

PyTorch provides device memory and streams; every computation runs in the
library's CUDA kernels.  All functions take device tensors and enqueue on the
current (or given) CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import MSA_DNA, MSA_PROTEIN, SeqSetC


class MsaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"msa status {code}: {msg}")
        self.code = code


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


class Context:
    """Owns the library context: device workspace and the autotune table."""

    def __init__(self, device: int = 0, workspace_bytes: int = 1 << 30):
        torch.cuda.init()
        self.device = device
        self._h = ctypes.c_void_p()
        with torch.cuda.device(device):
            rc = _lib.lib().msa_ctx_create(ctypes.byref(self._h), device, int(workspace_bytes))
        if rc != 0:
            raise MsaError(rc, "msa_ctx_create failed")

    @property
    def handle(self):
        return self._h

    def error(self) -> str:
        return _lib.lib().msa_last_error(self._h).decode()

    def raise_if(self, rc: int):
        if rc != 0:
            raise MsaError(rc, self.error())

    def check(self, stream=None):
        """Synchronise the stream and raise on any device-recorded error."""
        self.raise_if(_lib.lib().msa_ctx_check(self._h, _stream(stream)))

    def prof_enable(self, on: bool = True):
        self.raise_if(_lib.lib().msa_prof_enable(self._h, 1 if on else 0))

    def prof_read(self, reset: bool = True):
        """(summed DP-kernel milliseconds, kernels launched) since the last reset."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int64(0)
        self.raise_if(_lib.lib().msa_prof_read(self._h, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0))
        return ms.value, n.value

    def close(self):
        if self._h:
            _lib.lib().msa_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ALPHA = {"dna": MSA_DNA, "protein": MSA_PROTEIN}


class DeviceSeqs:
    """A sequence set resident on the GPU: ASCII arena, offsets, and the
    packed codes / bit planes written by :func:`pack`."""

    def __init__(self, ascii: torch.Tensor, offs: torch.Tensor, alphabet: str, max_len: int, total: int):
        self.alphabet = alphabet
        self.alpha = _ALPHA[alphabet]
        self.ascii = ascii
        self.offs = offs
        self.n = offs.numel() - 1
        self.total = int(total)
        self.max_len = int(max_len)
        L = _lib.lib()
        self.codes = torch.empty(int(L.msa_code_bytes(self.total)), dtype=torch.uint8, device=ascii.device)
        self.planes = torch.empty(int(L.msa_plane_words(self.total, self.alpha)), dtype=torch.int32,
                                  device=ascii.device)
        self.c = SeqSetC(_ptr(ascii), _ptr(offs), _ptr(self.codes), _ptr(self.planes), self.total,
                         self.n, self.alpha, self.max_len, 0)

    @staticmethod
    def from_host(arena: np.ndarray, offs: np.ndarray, alphabet: str = "dna", device="cuda",
                  pinned: bool = False) -> "DeviceSeqs":
        """Copy a host arena (``synth.SeqSet`` layout) to the device (H2D only)."""
        total = int(offs[-1]) if len(offs) else 0
        buf = np.zeros(max(16, (total + 15) // 16 * 16), dtype=np.uint8)
        buf[:total] = arena[:total]
        a = torch.from_numpy(buf)
        o = torch.from_numpy(np.ascontiguousarray(offs, dtype=np.int64))
        if pinned:
            a, o = a.pin_memory(), o.pin_memory()
        lens = np.diff(offs)
        max_len = int(lens.max()) if len(lens) else 0
        return DeviceSeqs(a.to(device, non_blocking=pinned), o.to(device, non_blocking=pinned),
                          alphabet, max_len, total)


def pack(ctx: Context, seqs: DeviceSeqs, stream=None) -> DeviceSeqs:
    """A1: ASCII -> byte codes + bit planes (msa_pack)."""
    ctx.raise_if(_lib.lib().msa_pack(ctx.handle, ctypes.byref(seqs.c), _stream(stream)))
    return seqs


def upload_and_pack(ctx: Context, ds, stream=None, pinned=False) -> DeviceSeqs:
    """Copy a ``synth.SeqSet`` to the device and pack it."""
    seqs = DeviceSeqs.from_host(ds.arena, ds.offs, ds.alphabet, pinned=pinned)
    return pack(ctx, seqs, stream)


def _pairs_tensor(pairs) -> torch.Tensor:
    if isinstance(pairs, np.ndarray):
        pairs = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32))
    if pairs.device.type != "cuda":
        pairs = pairs.cuda()
    return pairs.contiguous().view(-1, 2)


def lev_batch(ctx: Context, seqs: DeviceSeqs, pairs, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """A2/A3: Levenshtein distance of every pair (msa_lev_batch); int32 [P]."""
    pairs = _pairs_tensor(pairs)
    P = pairs.shape[0]
    if out is None:
        out = torch.empty(P, dtype=torch.int32, device=pairs.device)
    ctx.raise_if(_lib.lib().msa_lev_batch(ctx.handle, ctypes.byref(seqs.c), _ptr(pairs), P, _ptr(out),
                                          _stream(stream)))
    return out


def lev_one_to_many(ctx: Context, seqs: DeviceSeqs, query: int, idx, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Distances from sequence ``query`` to every sequence of ``idx``
    (msa_lev_one_to_many); int32 [n]."""
    if not isinstance(idx, torch.Tensor):
        idx = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32))
    idx = idx.to(device="cuda", dtype=torch.int32).contiguous()
    n = idx.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=idx.device)
    ctx.raise_if(_lib.lib().msa_lev_one_to_many(ctx.handle, ctypes.byref(seqs.c), int(query), _ptr(idx), n,
                                                _ptr(out), _stream(stream)))
    return out


def lev_banded_batch(ctx: Context, seqs: DeviceSeqs, pairs, k0, out: torch.Tensor | None = None,
                     k_used: torch.Tensor | None = None, stream=None):
    """A4: exact distances by certified Ukkonen bands starting at ``k0``.

    Returns ``(d[P], k_used[P])`` (int32).
    """
    pairs = _pairs_tensor(pairs)
    P = pairs.shape[0]
    if isinstance(k0, np.ndarray):
        k0 = torch.from_numpy(np.ascontiguousarray(k0, dtype=np.int32))
    k0 = k0.to(device=pairs.device, dtype=torch.int32).contiguous()
    if out is None:
        out = torch.empty(P, dtype=torch.int32, device=pairs.device)
    if k_used is None:
        k_used = torch.empty(P, dtype=torch.int32, device=pairs.device)
    ctx.raise_if(_lib.lib().msa_lev_banded_batch(ctx.handle, ctypes.byref(seqs.c), _ptr(pairs), P, _ptr(k0),
                                                 _ptr(out), _ptr(k_used), _stream(stream)))
    return out, k_used


class ByteSeqs:
    """Byte strings on the device for NW: ``codes[offs[s]:offs[s+1]]``."""

    def __init__(self, codes: torch.Tensor, offs: torch.Tensor, max_len: int, total: int | None = None):
        self.codes = codes
        self.offs = offs
        self.n = offs.numel() - 1
        self.max_len = int(max_len)
        self.total = int(codes.numel()) if total is None else int(total)

    @staticmethod
    def from_device_seqs(seqs: "DeviceSeqs") -> "ByteSeqs":
        return ByteSeqs(seqs.codes, seqs.offs, seqs.max_len, seqs.total)

    @staticmethod
    def from_list(rows, device="cuda") -> "ByteSeqs":
        lens = np.array([len(r) for r in rows], np.int64)
        offs = np.zeros(len(rows) + 1, np.int64)
        np.cumsum(lens, out=offs[1:])
        arena = np.frombuffer(b"".join(bytes(r) for r in rows) + b"\0", np.uint8).copy()
        return ByteSeqs(torch.from_numpy(arena).to(device), torch.from_numpy(offs).to(device),
                        int(lens.max()) if len(lens) else 0, int(offs[-1]))


def nw_align_batch(ctx: Context, seqs, pairs, match=0, mismatch=1, gap=1, ops_off: torch.Tensor | None = None,
                   stream=None, gap_open: int | None = None, ops: torch.Tensor | None = None,
                   sub: torch.Tensor | None = None):
    """A5/A6: NW score, edit script (forward order, bytes M/X/D/I) per pair.

    Returns ``(score[P] int32, ops uint8, ops_off[P+1] int64, ops_len[P] int32)``.
    ``seqs`` is a :class:`ByteSeqs` or a packed :class:`DeviceSeqs` (its byte codes).
    With ``gap_open`` the gap costs are affine: a run of L gaps costs
    ``gap_open + L * gap`` (msa_nw_align_batch_affine); with ``sub`` as well
    (device int32 [nsym, nsym] costs by code, e.g. :func:`blosum62_table`) a
    substitution costs ``sub[a, b]`` (msa_nw_align_batch_affine_sub).  A
    caller that passes both ``ops_off`` and an ``ops`` buffer of
    ``ops_off[-1]`` bytes makes the call without a host synchronisation.
    """
    if isinstance(seqs, DeviceSeqs):
        seqs = ByteSeqs.from_device_seqs(seqs)
    pairs = _pairs_tensor(pairs)
    P = pairs.shape[0]
    dev = pairs.device
    if ops_off is None:
        lens = seqs.offs[1:] - seqs.offs[:-1]
        cap = lens[pairs[:, 0].long()] + lens[pairs[:, 1].long()]
        ops_off = torch.zeros(P + 1, dtype=torch.int64, device=dev)
        torch.cumsum(cap, 0, out=ops_off[1:])
    if ops is None:                      # sized from the offsets (one device read)
        cap_total = int(ops_off[-1].item()) if P else 0
        ops = torch.empty(max(cap_total, 1), dtype=torch.uint8, device=dev)
    score = torch.empty(P, dtype=torch.int32, device=dev)
    ops_len = torch.empty(P, dtype=torch.int32, device=dev)
    if gap_open is None:
        ctx.raise_if(_lib.lib().msa_nw_align_batch(ctx.handle, _ptr(seqs.codes), _ptr(seqs.offs), seqs.n, seqs.total,
                                                   seqs.max_len, _ptr(pairs), P, match, mismatch, gap, _ptr(score),
                                                   _ptr(ops), _ptr(ops_off), _ptr(ops_len), _stream(stream)))
    elif sub is None:
        ctx.raise_if(_lib.lib().msa_nw_align_batch_affine(
            ctx.handle, _ptr(seqs.codes), _ptr(seqs.offs), seqs.n, seqs.total, seqs.max_len, _ptr(pairs), P, match,
            mismatch, gap_open, gap, _ptr(score), _ptr(ops), _ptr(ops_off), _ptr(ops_len), _stream(stream)))
    else:
        sub = sub.to(device=dev, dtype=torch.int32).contiguous()
        ctx.raise_if(_lib.lib().msa_nw_align_batch_affine_sub(
            ctx.handle, _ptr(seqs.codes), _ptr(seqs.offs), seqs.n, seqs.total, seqs.max_len, _ptr(pairs), P,
            _ptr(sub), int(sub.shape[0]), gap_open, gap, _ptr(score), _ptr(ops), _ptr(ops_off), _ptr(ops_len),
            _stream(stream)))
    return score, ops, ops_off, ops_len


def nw_align_batch_anchored(ctx: Context, seqs, pairs, k=12, match=0, mismatch=1, gap=1,
                            ops_off: torch.Tensor | None = None, stream=None, gap_open: int | None = None,
                            sub: torch.Tensor | None = None):
    """NW split at unique k-mer anchors (msa_nw_align_batch_anchored):
    runs of matches along the chained anchors, NW on the segments between
    them.  With ``gap_open`` the segments take affine gaps (``gap`` is the
    extension; msa_nw_align_batch_anchored_affine), with ``sub`` as well a
    substitution table (msa_nw_align_batch_anchored_affine_sub).  Returns
    ``(score[P] int32, ops uint8, ops_off[P+1] int64, ops_len[P] int32)``
    like :func:`nw_align_batch`."""
    if isinstance(seqs, DeviceSeqs):
        seqs = ByteSeqs.from_device_seqs(seqs)
    pairs = _pairs_tensor(pairs)
    P = pairs.shape[0]
    dev = pairs.device
    if ops_off is None:
        lens = seqs.offs[1:] - seqs.offs[:-1]
        cap = lens[pairs[:, 0].long()] + lens[pairs[:, 1].long()]
        ops_off = torch.zeros(P + 1, dtype=torch.int64, device=dev)
        torch.cumsum(cap, 0, out=ops_off[1:])
    cap_total = int(ops_off[-1].item()) if P else 0
    ops = torch.empty(max(cap_total, 1), dtype=torch.uint8, device=dev)
    score = torch.empty(P, dtype=torch.int32, device=dev)
    ops_len = torch.empty(P, dtype=torch.int32, device=dev)
    L = _lib.lib()
    if gap_open is None:
        ctx.raise_if(L.msa_nw_align_batch_anchored(
            ctx.handle, _ptr(seqs.codes), _ptr(seqs.offs), seqs.n, seqs.total, seqs.max_len, _ptr(pairs), P, k,
            match, mismatch, gap, _ptr(score), _ptr(ops), _ptr(ops_off), _ptr(ops_len), _stream(stream)))
    elif sub is None:
        ctx.raise_if(L.msa_nw_align_batch_anchored_affine(
            ctx.handle, _ptr(seqs.codes), _ptr(seqs.offs), seqs.n, seqs.total, seqs.max_len, _ptr(pairs), P, k,
            match, mismatch, gap_open, gap, _ptr(score), _ptr(ops), _ptr(ops_off), _ptr(ops_len), _stream(stream)))
    else:
        sub = sub.to(device=dev, dtype=torch.int32).contiguous()
        ctx.raise_if(L.msa_nw_align_batch_anchored_affine_sub(
            ctx.handle, _ptr(seqs.codes), _ptr(seqs.offs), seqs.n, seqs.total, seqs.max_len, _ptr(pairs), P, k,
            _ptr(sub), int(sub.shape[0]), gap_open, gap, _ptr(score), _ptr(ops), _ptr(ops_off), _ptr(ops_len),
            _stream(stream)))
    return score, ops, ops_off, ops_len


def blosum62_table(device="cuda") -> torch.Tensor:
    """BLOSUM62 as costs (-score) over the protein codes 0..19 and the gap
    code 20 of gapped centre rows: int32 [21, 21] (see ``substitution``)."""
    from . import substitution
    return torch.tensor(substitution.blosum62_costs_by_code(), dtype=torch.int32, device=device)


def lev_schedule(ctx: Context, lane_min_targets: int = -1, slot_min_targets: int = -1, lane_per_task: int = -1,
                 warp_per_task: int = -1) -> dict:
    """Sets the entries of msa_lev_batch's schedule that are given (>= 0;
    see ``msa_lev_tune_set``) and returns the schedule in force."""
    v = (ctypes.c_int32 * 4)(lane_min_targets, slot_min_targets, lane_per_task, warp_per_task)
    if any(x >= 0 for x in v):
        ctx.raise_if(_lib.lib().msa_lev_tune_set(ctx.handle, v))
    ctx.raise_if(_lib.lib().msa_lev_tune_get(ctx.handle, v))
    return dict(lane_min_targets=v[0], slot_min_targets=v[1], lane_per_task=v[2], warp_per_task=v[3])


def lev_autotune(ctx: Context, seqs: DeviceSeqs, pairs, out: torch.Tensor | None = None, stream=None):
    """A7: choose the schedule for batches like this one; returns the distances."""
    pairs = _pairs_tensor(pairs)
    P = pairs.shape[0]
    if out is None:
        out = torch.empty(P, dtype=torch.int32, device=pairs.device)
    ctx.raise_if(_lib.lib().msa_lev_autotune(ctx.handle, ctypes.byref(seqs.c), _ptr(pairs), P, _ptr(out),
                                             _stream(stream)))
    return out


# ---------------------------------------------------------------------------
# learned band proposer (A8-A10)
# ---------------------------------------------------------------------------

MLP_SHAPES = (("W1", (128, 256)), ("b1", (128,)), ("W2", (64, 128)), ("b2", (64,)), ("W3", (64,)), ("b3", (1,)))


def mlp_init_params(seed: int = 0) -> dict:
    """He-initialised parameters (numpy float32), in the library's layout."""
    rng = np.random.default_rng(seed)
    return dict(W1=(rng.standard_normal((128, 256)) * np.sqrt(2 / 256)).astype(np.float32),
                b1=np.zeros(128, np.float32),
                W2=(rng.standard_normal((64, 128)) * np.sqrt(2 / 128)).astype(np.float32),
                b2=np.zeros(64, np.float32),
                W3=(rng.standard_normal(64) * np.sqrt(1 / 64)).astype(np.float32),
                b3=np.zeros(1, np.float32))


def flatten_params(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], np.float32).reshape(-1) for k, _ in MLP_SHAPES])


def unflatten_params(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for k, shp in MLP_SHAPES:
        n = int(np.prod(shp))
        out[k] = flat[o:o + n].reshape(shp)
        o += n
    return out


class BandModel:
    """Device state of the band-proposer network (parameters, Adam moments)."""

    def __init__(self, ctx: Context, params: dict | None = None, seed: int = 0):
        L = _lib.lib()
        self.ctx = ctx
        self.np = int(L.msa_mlp_num_params())
        self.state = torch.zeros(int(L.msa_mlp_state_bytes()) // 4, dtype=torch.float32, device="cuda")
        self.set_params(params if params is not None else mlp_init_params(seed))

    def set_params(self, params: dict, stream=None):
        flat = torch.from_numpy(flatten_params(params)).cuda()
        assert flat.numel() == self.np
        self.state[: self.np].copy_(flat)
        self.ctx.raise_if(_lib.lib().msa_mlp_sync(self.ctx.handle, _ptr(self.state), _stream(stream)))

    def params(self) -> dict:
        return unflatten_params(self.state[: self.np].cpu().numpy().copy())

    def forward(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        P = X.shape[0]
        y = torch.empty(P, dtype=torch.float32, device=X.device)
        self.ctx.raise_if(_lib.lib().msa_mlp_forward(self.ctx.handle, _ptr(self.state), _ptr(X), P, _ptr(y),
                                                     _stream(stream)))
        return y

    def train_step(self, X: torch.Tensor, y: torch.Tensor, idx: torch.Tensor, lr: float, tau: float = 0.9,
                   stream=None) -> torch.Tensor:
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        self.ctx.raise_if(_lib.lib().msa_mlp_train_step(self.ctx.handle, _ptr(self.state), _ptr(X), _ptr(y),
                                                        int(X.shape[0]), _ptr(idx), int(idx.numel()), float(lr),
                                                        float(tau),
                                                        _ptr(loss), _stream(stream)))
        return loss

    def read_grad(self, stream=None) -> dict:
        g = torch.empty(self.np, dtype=torch.float32, device="cuda")
        self.ctx.raise_if(_lib.lib().msa_mlp_read_grad(self.ctx.handle, _ptr(self.state), _ptr(g), _stream(stream)))
        return unflatten_params(g.cpu().numpy())

    def calibrate(self, yhat: torch.Tensor, y: torch.Tensor, tau: float = 0.95, stream=None):
        """Fits the band calibration from held-out network outputs and true
        y = f / max(m, n) (device fp32); ``calibrate(None, None)`` removes it."""
        N = 0 if yhat is None else int(yhat.numel())
        if N:
            assert y.numel() == N and yhat.dtype == torch.float32 and y.dtype == torch.float32
        self.ctx.raise_if(_lib.lib().msa_band_calibrate(self.ctx.handle, _ptr(self.state),
                                                        _ptr(yhat) if N else None, _ptr(y) if N else None, N,
                                                        float(tau), _stream(stream)))

    def calibration(self):
        """The 33 calibration knots, or None when the state holds none."""
        cal = self.state[-64:].cpu().numpy()
        return cal[1:34].copy() if cal[0] != 0 else None

    def predict_band(self, seqs: DeviceSeqs, prof: torch.Tensor, pairs, gamma: float = 0.1, margin: int = 8,
                     stream=None):
        """Fused features + forward + band policy: returns ``(yhat[P], k[P])``."""
        pairs = _pairs_tensor(pairs)
        P = pairs.shape[0]
        yhat = torch.empty(P, dtype=torch.float32, device=pairs.device)
        k = torch.empty(P, dtype=torch.int32, device=pairs.device)
        self.ctx.raise_if(_lib.lib().msa_band_predict(self.ctx.handle, _ptr(self.state), ctypes.byref(seqs.c),
                                                      _ptr(prof), _ptr(pairs), P, float(gamma), int(margin),
                                                      _ptr(yhat), _ptr(k), _stream(stream)))
        return yhat, k


def kmer_profile(ctx: Context, seqs: DeviceSeqs, stream=None) -> torch.Tensor:
    """A8: uint16 [n][256] 4-mer counts (returned as int16 storage)."""
    prof = torch.empty((seqs.n, 256), dtype=torch.int16, device="cuda")
    ctx.raise_if(_lib.lib().msa_kmer_profile(ctx.handle, ctypes.byref(seqs.c), _ptr(prof), _stream(stream)))
    return prof


def pair_features(ctx: Context, seqs: DeviceSeqs, prof: torch.Tensor, pairs, stream=None) -> torch.Tensor:
    """bf16 [P][256] pair features (as bfloat16 tensor)."""
    pairs = _pairs_tensor(pairs)
    P = pairs.shape[0]
    X = torch.empty((P, 256), dtype=torch.bfloat16, device="cuda")
    ctx.raise_if(_lib.lib().msa_pair_features(ctx.handle, ctypes.byref(seqs.c), _ptr(prof), _ptr(pairs), P,
                                              _ptr(X), _stream(stream)))
    return X


# ---------------------------------------------------------------------------
# guide tree (A11) and merge (A12)
# ---------------------------------------------------------------------------

class Tree:
    """Cluster tree of Alg. 1: ``order`` (device) and host node arrays in BFS order."""

    def __init__(self, n: int):
        cap = max(1, 2 * n - 1)
        self.n = n
        self.order = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        self.lo, self.hi, self.center, self.left, self.right, self.parent = (
            np.full(cap, -1, np.int32) for _ in range(6))
        self.n_nodes = 0

    def members(self, k: int, order_host: np.ndarray | None = None) -> list:
        o = self.order.cpu().numpy() if order_host is None else order_host
        return sorted(int(x) for x in o[self.lo[k]:self.hi[k]])


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def clam_partition(ctx: Context, seqs: DeviceSeqs, band: "BandModel | None" = None, prof: torch.Tensor | None = None,
                   gamma: float = 0.2, margin: int = 8, stream=None) -> Tree:
    """A11: build the guide tree (msa_clam_partition).

    With ``band`` (a trained :class:`BandModel`) the distance batches start
    from the network's bands (msa_clam_partition_banded); the tree is the same.
    """
    t = Tree(seqs.n)
    nn = ctypes.c_int32(0)
    outs = (_ptr(t.order), _np_ptr(t.lo), _np_ptr(t.hi), _np_ptr(t.center), _np_ptr(t.left), _np_ptr(t.right),
            _np_ptr(t.parent), ctypes.byref(nn), _stream(stream))
    if band is None:
        ctx.raise_if(_lib.lib().msa_clam_partition(ctx.handle, ctypes.byref(seqs.c), *outs))
    else:
        if prof is None:
            prof = kmer_profile(ctx, seqs, stream)
        ctx.raise_if(_lib.lib().msa_clam_partition_banded(ctx.handle, ctypes.byref(seqs.c), _ptr(band.state),
                                                          _ptr(prof), gamma, margin, *outs))
    t.n_nodes = nn.value
    return t


def merge_tree(ctx: Context, seqs: DeviceSeqs, tree: Tree, match=0, mismatch=1, gap=1, stream=None,
               gap_open: int | None = None, sub: torch.Tensor | None = None):
    """A12: bottom-up merge; returns ``(pos tensor, width[n_nodes], score[n_nodes])``.

    With ``gap_open`` the center alignments use affine gaps (a run of L gaps
    costs ``gap_open + L * gap``; msa_merge_tree_affine), and with ``sub``
    (device int32 [nsym, nsym] covering the gap code) substitutions cost
    ``sub[a, b]`` (msa_merge_tree_affine_sub)."""
    pos = torch.empty(max(seqs.total, 1), dtype=torch.int32, device="cuda")
    width = np.zeros(max(tree.n_nodes, 1), np.int32)
    score = np.zeros(max(tree.n_nodes, 1), np.int32)
    tr = (ctypes.byref(seqs.c), _ptr(tree.order), _np_ptr(tree.lo), _np_ptr(tree.hi), _np_ptr(tree.center),
          _np_ptr(tree.left), _np_ptr(tree.right), tree.n_nodes, match, mismatch)
    outs = (_ptr(pos), _np_ptr(width), _np_ptr(score), _stream(stream))
    if gap_open is None:
        ctx.raise_if(_lib.lib().msa_merge_tree(ctx.handle, *tr, gap, *outs))
    elif sub is None:
        ctx.raise_if(_lib.lib().msa_merge_tree_affine(ctx.handle, *tr, gap_open, gap, *outs))
    else:
        sub = sub.to(device="cuda", dtype=torch.int32).contiguous()
        ctx.raise_if(_lib.lib().msa_merge_tree_affine_sub(ctx.handle, *tr[:-2], _ptr(sub), int(sub.shape[0]),
                                                           gap_open, gap, *outs))
    return pos, width[: tree.n_nodes], score[: tree.n_nodes]


def msa_rows(ctx: Context, seqs: DeviceSeqs, tree: Tree, pos: torch.Tensor, W: int, stream=None) -> torch.Tensor:
    """The MSA as uint8 [n, W] rows in tree order (ASCII, '-' for gaps)."""
    rows = torch.empty((max(seqs.n, 1), max(W, 1)), dtype=torch.uint8, device="cuda")
    ctx.raise_if(_lib.lib().msa_msa_rows(ctx.handle, ctypes.byref(seqs.c), _ptr(tree.order), _ptr(pos), int(W),
                                         _ptr(rows), _stream(stream)))
    return rows[: seqs.n, :W]


def msa_metrics(ctx: Context, seqs: DeviceSeqs, tree: Tree, rows: torch.Tensor, sample: int | None = 10000,
                seed: int = 0, gap: int = ord("-"), stream=None) -> dict:
    """Alignment quality (section "Evaluation"; msa_msa_metrics) over a seeded
    random sample of ``sample`` rows (all rows when None or larger)."""
    R, W = rows.shape
    if sample is None or sample >= R:
        pick = np.arange(R)
    else:
        pick = np.sort(np.random.default_rng(seed).choice(R, size=sample, replace=False))
    order = tree.order.cpu().numpy()
    srows = torch.from_numpy(pick.astype(np.int32)).cuda()
    sseqs = torch.from_numpy(order[pick].astype(np.int32)).cuda()
    out = np.zeros(3, np.float64)
    cnt = np.zeros(4, np.int64)
    ctx.raise_if(_lib.lib().msa_msa_metrics(ctx.handle, ctypes.byref(seqs.c), _ptr(rows.contiguous()), R, W,
                                            _ptr(srows), _ptr(sseqs), len(pick), gap, _np_ptr(out), _np_ptr(cnt),
                                            _stream(stream)))
    return dict(pct_gaps=float(out[0]), p_score=float(out[1]), distortion=float(out[2]), rows=int(len(pick)),
                gaps=int(cnt[0]), compared=int(cnt[1]), mismatched=int(cnt[2]), pairs=int(cnt[3]), sample=pick)


# ---------------------------------------------------------------------------
# measurement
# ---------------------------------------------------------------------------

PROBE_OPS = {"lop3": 0, "shf": 1, "addc": 2, "word_step": 3, "imad": 4}


def probe_int_pipe(ctx: Context, op: str, iters: int = 4096, reps: int = 3, stream=None) -> dict:
    """Measured throughput of one integer operation kind (msa_probe_int_pipe):
    the best of ``reps`` timed launches after a warm-up, in lane-ops/s."""
    code = PROBE_OPS[op]
    n = ctypes.c_int64(0)
    st = _stream(stream)
    ctx.raise_if(_lib.lib().msa_probe_int_pipe(ctx.handle, code, int(iters), ctypes.byref(n), st))
    best = float("inf")
    cur = torch.cuda.current_stream() if stream is None else stream
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        ctx.raise_if(_lib.lib().msa_probe_int_pipe(ctx.handle, code, int(iters), ctypes.byref(n), st))
        b.record(cur)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return dict(op=op, lane_ops=int(n.value), ms=best, ops_per_s=n.value / (best / 1e3))
