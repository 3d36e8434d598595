"""The 5-slice mixed path's launch schedule (the sequence launch_mixed_steps
issues, restated here): panels in groups of four; before panel J is factored
its tile column's data rows receive the group's earlier panels; after it the
right-hand-side row receives panel J; after the group the data triangle beyond
it receives all of the group's panels in one item (K = 4 x 128 at most, the
limit of the exact FP32 accumulators).  Checked for every tile count nb the
workloads reach and beyond: every trailing tile receives every earlier panel
exactly once, in panel order, before its own column is factored (the
right-looking Cholesky of the bordered matrix, Section 3.3 Step 3); and every
panel image an item reads is still in the panel slot it was written to (four
slots per tile row, panel J in slot J % 4)."""
import pytest

GP = 4


def schedule(nb):
    """The launches of one 5-slice pass over nb data tile rows (tile row nb is
    the right-hand-side row): ('factor', J) or ('trail', mode, Klo, Ihi, P, J0),
    the item of mode 0 / 1 applying panels J0 .. J0 + P - 1, of mode 2 panel J0."""
    out = []
    for J0 in range(0, nb, GP):
        G = min(GP, nb - J0)
        Jend = J0 + G
        for J in range(J0, Jend):
            if J > J0:
                out.append(("trail", 1, J, nb - 1, J - J0, J0))
            out.append(("factor", J))
            out.append(("trail", 2, J + 1, nb, 1, J))
        out.append(("trail", 0, Jend, nb - 1, G, J0))
    return out


def items(mode, Klo, Ihi):
    """Tiles (I, K) of one launch: 0 the triangle Klo <= K <= I <= Ihi, 1 the
    column K = Klo, 2 the row I = Ihi."""
    if mode == 0:
        return [(I, K) for K in range(Klo, Ihi + 1) for I in range(K, Ihi + 1)]
    if mode == 1:
        return [(I, Klo) for I in range(Klo, Ihi + 1)]
    return [(Ihi, K) for K in range(Klo, Ihi + 1)]


def simulate(nb):
    applied = {(I, K): [] for K in range(nb + 1) for I in range(K, nb + 1)}
    slot = {}          # (tile row, slot) -> panel whose image it holds
    factored = []
    for op in schedule(nb):
        if op[0] == "factor":
            J = op[1]
            # the diagonal tile and every tile below it have all earlier panels
            for I in range(J, nb + 1):
                assert applied[(I, J)] == list(range(J)), (nb, "factor", J, I, applied[(I, J)])
            factored.append(J)
            # the panel solve writes the images of L_IJ, I = J + 1 .. nb (and
            # the diagonal tile's own) into slot J % 4 of each tile row
            for I in range(J, nb + 1):
                slot[(I, J % 4)] = J
            continue
        _, mode, Klo, Ihi, P, J0 = op
        assert 1 <= P <= GP
        if Ihi < Klo:
            continue
        panels = list(range(J0, J0 + P))
        assert all(p in factored for p in panels)
        for I, K in items(mode, Klo, Ihi):
            for p in panels:
                # operand images of rows I and K for panel p, still in their slots
                assert slot.get((I, p % 4)) == p and slot.get((K, p % 4)) == p, (nb, op, I, K, p)
                applied[(I, K)].append(p)
    return applied, factored


@pytest.mark.parametrize("nb", range(1, 70))
def test_every_update_once_in_order_before_its_column(nb):
    applied, factored = simulate(nb)
    assert factored == list(range(nb))
    for (I, K), got in applied.items():
        # tile (I, K) receives the panels J < K; the right-hand-side row and the
        # corner tile (nb, nb) receive every panel
        assert got == list(range(min(K, nb))), (nb, I, K, got)


def test_item_counts_of_a_step():
    """Half-tile items of the data triangle and columns, whole tiles of the
    right-hand-side row (its transposed form) at n = 4000 (nb = 32): the
    per-panel trailing tiles m (m + 1) / 2, m = nb - J, are all covered."""
    nb = 32
    tiles = 0
    for op in schedule(nb):
        if op[0] == "trail":
            _, mode, Klo, Ihi, P, _ = op
            tiles += len(items(mode, Klo, Ihi)) * P
    assert tiles == sum((nb - J) * (nb - J + 1) // 2 for J in range(nb))
