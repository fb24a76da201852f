"""Shared helpers of the GPU parity tests: oracle runs (cached) and the parity bar.

The bar (exact methods): every receiver-step that the oracle does not classify as near a
shadow boundary (status flips when the sun direction is rotated by 1e-4 rad along its
arc) must agree bit for bit; receivers with no near-boundary step must have equal gross
and continuous counts; and |gross difference| <= 1 on at least 99.9% of all receivers.
"""
from __future__ import annotations

import functools

import numpy as np

import oracle
from synth import configs

EPS_RAD = 1e-4


@functools.lru_cache(maxsize=None)
def workload(name: str, **kw):
    return configs.BY_NAME[name](**kw)


def oracle_bits(w, part: str, sample=None):
    """(bits [R,S], near [R,S]) for the ground ('ground') or facade ('facade') receivers."""
    if part == "ground":
        pos, nrm = w.ground.positions(), None
    else:
        pos, nrm = w.facade_pos, w.facade_nrm
    if sample is not None:
        pos = pos[sample]
        nrm = None if nrm is None else nrm[sample]
    t9, tb = w.mesh.tri9(), w.mesh.tri_building
    bits = oracle.shadow_bits(t9, tb, pos, nrm, w.sun.dirs)
    near = oracle.near_boundary(t9, tb, pos, nrm, w.sun.dirs, w.sun.day_start, bits, eps=EPS_RAD)
    return bits, near


_cache = {}


def cached_oracle(key, w, part, sample=None):
    if key not in _cache:
        _cache[key] = oracle_bits(w, part, sample)
    return _cache[key]


def assert_counts_parity(gross, cont, bits, near, day_start, label=""):
    og, oc = oracle.reduce(bits, day_start)
    strict = ~near.any(axis=1)
    bad = np.nonzero(strict & (gross != og))[0]
    assert bad.size == 0, f"{label}: {bad.size} strict receivers differ in gross, e.g. {bad[:5]}"
    if cont is not None:
        badc = np.nonzero(strict & (cont != oc))[0]
        assert badc.size == 0, f"{label}: {badc.size} strict receivers differ in continuous"
    within = np.abs(gross.astype(np.int64) - og) <= 1
    assert within.mean() >= 0.999, f"{label}: only {within.mean():.5f} within one step"
    return strict.mean()


def assert_bits_parity(gbits, bits, near, label=""):
    diff = (gbits != bits) & (near == 0)
    n = int(diff.sum())
    assert n == 0, f"{label}: {n} receiver-steps away from a boundary differ, e.g. {np.argwhere(diff)[:5].tolist()}"


def block_sizes(day_start, block_len: int = 0):
    """Block lengths of the library's partition of the sun table (sa_block_partition)."""
    from paper_1907_04435_gb300 import binding as B
    return B.block_partition(day_start, block_len)[1].tolist()


def unpack_masks(masks, sizes) -> np.ndarray:
    """[n_blocks, R] step masks (bit k = step k of the block, as sa_shadow_masks writes
    them) -> uint8 [R, S] per-step bits in block order."""
    mk = masks.cpu().numpy().view(np.uint64)
    R = mk.shape[1]
    cols = []
    for b, K in enumerate(sizes):
        bits = (mk[b][:, None] >> np.arange(K, dtype=np.uint64)[None, :]) & np.uint64(1)
        cols.append(bits.astype(np.uint8))
    return np.concatenate(cols, axis=1) if cols else np.zeros((R, 0), np.uint8)
