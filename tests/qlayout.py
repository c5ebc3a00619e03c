"""Decoder of the quantised tile layout declared in include/b3t.h (test
helper): 16 KiB chunks of 128 rows x 128 bytes, chunk (rb, kb) at
(rb * nk + kb) * 16384, row r at r * 128, 16-byte group g at g ^ (r % 8),
then the int32 scale exponent."""
import numpy as np
import torch


def decode(qbytes, b, fmt):
    """Q bytes (numpy uint8) -> (values as float64 (b x b, [r, c]), e)."""
    es = 2 if fmt == 0 else 1
    cpc = 128 // es
    nk = b // cpc
    data = qbytes[: b * b * es]
    e = int(np.frombuffer(qbytes[b * b * es: b * b * es + 4].tobytes(), dtype=np.int32)[0])
    out = np.empty((b, b))
    chunks = data.reshape(b // 128, nk, 128, 8, 16)   # rb, kb, row, group, byte
    for rb in range(b // 128):
        for kb in range(nk):
            ch = chunks[rb, kb]
            rows = np.arange(128)
            for g in range(8):
                pos = g ^ (rows % 8)
                grp = ch[rows, pos]                  # (128, 16) bytes of group g
                if es == 2:
                    bits = grp.view(np.uint16).astype(np.uint32) << 16
                    vals = bits.view(np.float32).astype(np.float64)
                else:
                    vals = torch.from_numpy(grp.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
                G = 16 // es
                c0 = kb * cpc + g * G
                out[rb * 128:(rb + 1) * 128, c0:c0 + G] = vals
    return out, e
