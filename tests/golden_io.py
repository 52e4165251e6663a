"""Readers for the hand-worked fixtures in tests/golden/ (no arithmetic)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_dark_channel_fixture(name="dark_channel_4x5.txt"):
    rgb_rows, m, D3, selects = [], None, None, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            if key == "rgb":
                rgb_rows.append([[int(v) for v in tri.split(",")] for tri in val.split()])
            elif key in ("m", "D3"):
                arr = np.array([[int(v) for v in row.split()] for row in val.split("|")], dtype=np.uint8)
                if key == "m":
                    m = arr
                else:
                    D3 = arr
            elif key == "select":
                toks = val.split()
                patch, K, T, n_above, cut = (int(v) for v in toks[:5])
                i_idx, i_S = toks.index("idx"), toks.index("S")
                idx = [int(v) for v in toks[i_idx + 1:i_S]]
                S = [int(v) for v in toks[i_S + 1:]]
                selects.append(dict(patch=patch, K=K, T=T, n_above=n_above,
                                    cut_index=cut, idx=idx, S=S))
    return np.array(rgb_rows, dtype=np.uint8), m, D3, selects
