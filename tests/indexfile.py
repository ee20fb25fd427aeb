"""Reader and writer of the index file format (test infrastructure).

Written from the format's description in include/adanns.h, independently of
the library: a 96-byte little-endian header (magic "ADANNSIX", version 1,
header size, N, d, d_c, nlist, metric, storage mask, OPQ d_s, OPQ M, a flag
word, reserved words), the FP32 centroids, the int32 list of every id, the
FP32 rows in id order, then with OPQ data the rotation, the codebooks and the
codes in id order.
"""
from __future__ import annotations

import struct

import numpy as np

HEADER = struct.Struct("<8sIIq8i10i")
assert HEADER.size == 96


def write(path, centroids, assign, rows, metric=1, storage=1, opq=None):
    """opq: None or dict(R [ds, ds], codebooks [M, 256, ds/M], codes [N, M] by id,
    optionally lcent [nlist, ds] for residual codes)."""
    centroids = np.ascontiguousarray(centroids, dtype="<f4")
    assign = np.ascontiguousarray(assign, dtype="<i4")
    rows = np.ascontiguousarray(rows, dtype="<f4")
    N, d = rows.shape
    nlist, d_c = centroids.shape
    ds = M = flags = 0
    if opq is not None:
        ds, M = opq["R"].shape[0], opq["codebooks"].shape[0]
        flags = 1 if opq.get("lcent") is not None else 0
    with open(path, "wb") as f:
        f.write(HEADER.pack(b"ADANNSIX", 1, 96, N, d, d_c, nlist, metric, storage, ds, M, flags,
                            *([0] * 10)))
        f.write(centroids.tobytes())
        f.write(assign.tobytes())
        f.write(rows.tobytes())
        if opq is not None:
            f.write(np.ascontiguousarray(opq["R"], dtype="<f4").tobytes())
            f.write(np.ascontiguousarray(opq["codebooks"], dtype="<f4").tobytes())
            f.write(np.ascontiguousarray(opq["codes"], dtype=np.uint8).tobytes())
            if flags:
                f.write(np.ascontiguousarray(opq["lcent"], dtype="<f4").tobytes())


def read(path):
    with open(path, "rb") as f:
        raw = f.read()
    h = HEADER.unpack_from(raw, 0)
    magic, version, hb, N, d, d_c, nlist, metric, storage, ds, M, flags = h[:12]
    out = {"magic": magic, "version": version, "header_bytes": hb, "N": N, "d": d, "d_c": d_c,
           "nlist": nlist, "metric": metric, "storage": storage, "opq_ds": ds, "opq_M": M,
           "opq_flags": flags}
    o = 96

    def take(dtype, count, shape):
        nonlocal o
        a = np.frombuffer(raw, dtype=dtype, count=count, offset=o).reshape(shape)
        o += a.nbytes
        return a

    out["centroids"] = take("<f4", nlist * d_c, (nlist, d_c))
    out["assign"] = take("<i4", N, (N,))
    out["rows"] = take("<f4", N * d, (N, d))
    if M:
        out["R"] = take("<f4", ds * ds, (ds, ds))
        out["codebooks"] = take("<f4", M * 256 * (ds // M), (M, 256, ds // M))
        out["codes"] = take(np.uint8, N * M, (N, M))
        if flags & 1:
            out["lcent"] = take("<f4", nlist * ds, (nlist, ds))
    out["trailing_bytes"] = len(raw) - o
    return out
