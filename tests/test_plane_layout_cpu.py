"""Host model of the shifted-plane sweep's store layout (no GPU).

The kernel stores node (x, y) of a finished plane at ((x - sx) mod nx,
(y - sy) mod ny) of the next step's frame, in the block that owns that stored
row, with a copy into the pad column (column 0 again, at nx) and into the halo
row of the band before (the first row of each band, or row 0 after the last
band).  The transaction-counted completion scheme (stage 3) lets each block
post, before the stores arrive, the bytes it will receive from other blocks:
per stored row (its band's rows and its halo row) nx + 1 node vectors when the
row's source row belongs to another block.  This test replays the kernel's
index arithmetic for every shift of many plane shapes and checks that every
stored position of every block (band rows, halo row, pad column) is written
exactly once and that each block's posted count equals what the other blocks
send; a wrong count would leave a wait to time out or a phase to complete
early.
"""

import pytest


def replay(nx, ny, nb, sx, sy):
    rows = -(-ny // nb)
    lastrows = ny - (nb - 1) * rows
    received = [0] * nb
    written = set()
    for sender in range(nb):
        y0 = sender * rows
        for q in range(min(rows, ny - y0) * nx):
            yl, x = divmod(q, nx)
            xs = (x - sx) % nx
            ys = (y0 + yl - sy) % ny
            ob = ys // rows
            lr = ys - ob * rows
            hb = nb - 1 if ob == 0 else ob - 1
            hr = lastrows if hb == nb - 1 else rows
            dests = [(ob, lr, xs)] + ([(ob, lr, nx)] if xs == 0 else [])
            if lr == 0:
                dests += [(hb, hr, xs)] + ([(hb, hr, nx)] if xs == 0 else [])
            for d in dests:
                assert d not in written, d
                written.add(d)
                if d[0] != sender:
                    received[d[0]] += 1
    for rank in range(nb):
        y0 = rank * rows
        myrows = min(rows, ny - y0)
        for r in range(myrows + 1):
            for c in range(nx + 1):
                assert (rank, r, c) in written, (rank, r, c)
        posted = 0
        for j in range(myrows + 1):
            ys = y0 + j if j < myrows else (0 if rank == nb - 1 else y0 + rows)
            if ((ys + sy) % ny) // rows != rank:
                posted += nx + 1
        assert posted == received[rank], (nx, ny, nb, sx, sy, rank)


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (8, 13), (12, 16), (5, 31)])
def test_every_position_once_and_counts_match(nx, ny):
    for nb in range(1, 17):
        rows = -(-ny // nb)
        if nb > ny or (nb - 1) * rows >= ny:
            continue
        for sx in range(nx):
            for sy in range(ny):
                replay(nx, ny, nb, sx, sy)
