"""Expected orbit-record layout of a periodic boundary grid, from first
principles (shared by the host-planning and the GPU parity tests)."""
from fractions import Fraction


def expected_slots(n1, n3, L1, L3, tile=128):
    """Member slots of the orbit layout: the half-spectrum bins grouped by their
    exact |k|^2 (rational arithmetic on the exact binary values of L1, L3), a
    Nyquist bin counting 2 members (the corner 4), each class packed into
    records of 4 without splitting a bin, records padded to whole tiles."""
    classes = {}
    for r3 in range(n3):
        j3 = r3 if r3 <= n3 // 2 else r3 - n3
        for j1 in range(n1 // 2 + 1):
            key = (Fraction(j1) / Fraction(L1)) ** 2 + (Fraction(j3) / Fraction(L3)) ** 2
            classes.setdefault(key, []).append((2 if j1 == n1 // 2 else 1) * (2 if r3 == n3 // 2 else 1))
    records = 0
    for sizes in classes.values():
        fill = 0
        for m in sizes:
            if fill + m > 4:
                records, fill = records + 1, 0
            fill += m
        records += 1
    return 4 * (-(-records // tile) * tile)


def square_grid_records(n, tile=128):
    """Orbit records of an n x n grid with equal spacings, in the layout's
    order: half-spectrum bins sorted by (j1^2 + j3^2, j1, r3), each class of
    equal |k| packed into records of 4 member slots without splitting a bin (a
    Nyquist bin takes 2 slots, the corner 4).  Returns (records, n_records
    padded to whole tiles); each record is a list of flat bins r3 (n/2+1) + j1."""
    import numpy as np
    nh = n // 2 + 1
    r3, j1 = np.meshgrid(np.arange(n), np.arange(nh), indexing="ij")
    r3, j1 = r3.ravel(), j1.ravel()
    j3 = np.where(r3 <= n // 2, r3, r3 - n)
    key = j1.astype(np.int64) ** 2 + j3.astype(np.int64) ** 2
    order = np.lexsort((r3, j1, key))
    slots = np.where(j1 == n // 2, 2, 1) * np.where(r3 == n // 2, 2, 1)
    records, cur, fill, last = [], [], 0, None
    for i in order:
        k = int(key[i])
        if last is not None and (k != last or fill + slots[i] > 4):
            records.append(cur)
            cur, fill = [], 0
        cur.append(int(r3[i] * nh + j1[i]))
        fill += int(slots[i])
        last = k
    records.append(cur)
    return records, -(-len(records) // tile) * tile
