"""Expected record layout of a periodic boundary grid, from first principles
(shared by the host-planning and the GPU parity tests).

The half-spectrum bins are grouped by their exact |k|^2 (integer keys
(j1 b)^2 + (j3 a)^2 for L1 / L3 = a / b, the exact ratio of the binary values
of L1 and L3) and ordered by (|k|^2, j1, r3).  A bin contributes 1 member slot,
2 on a Nyquist line and 4 at the corner.  Records have 4 slots in two halves of
2; the members of one bin share a record.

* whole records: each class fills records of its own;
* half records: each class fills halves (a Nyquist bin one half, the corner a
  record, other bins two to a half); a class's halves pair up into records and
  an odd leftover half pairs with the next class's leftover.

A grid uses whole records unless they exceed 1.03 x the bins in slots and
1.12 x the slots of the half records (the half-record kernels stream their
bytes ~13 % slower, so half records must save more than that).
"""
from fractions import Fraction


def _classes(n1, n3, L1, L3):
    """Classes of equal |k| in |k| order; each a list of (flat bin, slots)."""
    ratio = Fraction(L1) / Fraction(L3)
    a, b = ratio.numerator, ratio.denominator
    nh = n1 // 2 + 1
    items = []
    for r3 in range(n3):
        j3 = r3 if r3 <= n3 // 2 else r3 - n3
        for j1 in range(nh):
            key = (j1 * b) ** 2 + (j3 * a) ** 2
            slots = (2 if j1 == n1 // 2 else 1) * (2 if r3 == n3 // 2 else 1)
            items.append((key, j1, r3, r3 * nh + j1, slots))
    items.sort()
    classes, last = [], None
    for key, _, _, flat, slots in items:
        if key != last:
            classes.append([])
            last = key
        classes[-1].append((flat, slots))
    return classes


def _whole(classes):
    records = []
    for cls in classes:
        cur, fill = [], 0
        for flat, slots in cls:
            if fill + slots > 4:
                records.append(cur)
                cur, fill = [], 0
            cur.append(flat)
            fill += slots
        records.append(cur)
    return records


def _halves(classes):
    records, left = [], None
    for cls in classes:
        halves, singles = [], []
        for flat, slots in cls:
            if slots == 1:
                singles.append(flat)
            else:
                halves.extend([[flat]] * (slots // 2))
        halves += [singles[k:k + 2] for k in range(0, len(singles), 2)]
        h = 0
        while h + 1 < len(halves):
            records.append(sorted(set(halves[h] + halves[h + 1])))
            h += 2
        if h < len(halves):
            if left is None:
                left = halves[h]
            else:
                records.append(left + halves[h])
                left = None
    if left is not None:
        records.append(left)
    return records


def grid_records(n1, n3, L1, L3):
    """(records, halves): the records as lists of flat bins, in layout order."""
    classes = _classes(n1, n3, L1, L3)
    whole = _whole(classes)
    if 4 * len(whole) <= 1.03 * n3 * (n1 // 2 + 1):
        return whole, False
    halves = _halves(classes)
    if len(whole) <= 1.12 * len(halves):
        return whole, False
    return halves, True


def expected_slots(n1, n3, L1, L3, tile=128):
    """Member slots of the layout, records padded to whole tiles of 128."""
    records, _ = grid_records(n1, n3, L1, L3)
    return 4 * (-(-len(records) // tile) * tile)


def square_grid_records(n, tile=128):
    """Records of an n x n grid with equal spacings and their count padded to
    whole tiles (the layout of a square grid; integer keys j1^2 + j3^2)."""
    records, _ = grid_records(n, n, float(n), float(n))
    return records, -(-len(records) // tile) * tile
