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
