"""Test-side glue between oracle trees (dicts) and the library's node order."""
import numpy as np

from oracle import tree as OT


def spread3(v):
    out = 0
    for b in range(21):
        out |= ((v >> b) & 1) << (3 * b)
    return out


def morton(a1, a2, a3):
    return (spread3(a1) << 2) | (spread3(a2) << 1) | spread3(a3)


def oracle_to_arrays(tree, k):
    """Oracle tree dict -> (coords (n,4) int32, leaf (n,), blocks (n,k,k,k)),
    sorted by level then Morton key as the C ABI requires."""
    keys = sorted(tree.keys(), key=lambda key: (key[0], morton(*key[1:])))
    coords = np.array(keys, dtype=np.int32).reshape(-1, 4)
    leaf = np.array([tree[key].leaf for key in keys], dtype=np.int32)
    blocks = np.zeros((len(keys), k, k, k))
    for i, key in enumerate(keys):
        if tree[key].s is not None:
            blocks[i] = tree[key].s
    return coords, leaf, blocks


def arrays_to_dict(coords, blocks):
    return {tuple(int(v) for v in c): b for c, b in zip(coords, blocks)}


def rel_l2(a_dict, b_dict, keys=None):
    keys = keys if keys is not None else list(b_dict.keys())
    num = sum(float(((a_dict[key] - b_dict[key]) ** 2).sum()) for key in keys)
    den = sum(float((b_dict[key] ** 2).sum()) for key in keys)
    return (num / den) ** 0.5 if den > 0 else num ** 0.5


def oracle_density(d):
    return OT.Density(d.coef, d.expo, d.centers, d.r2coef)
