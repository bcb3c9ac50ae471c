"""The invariant behind the boundary update's phase A (host logic, no GPU).

Phase A pushes, from every source cell s, the population f+_i(s) into entry
(i, k) of the listed cell k = s + c_i when that cell is FLUID_BOUNDARY, and, when
s is itself listed, f+_opp(i)(s) into entry (i, k_s) for each of its solid links
i.  Phase B then reads entry (i, k) as the population that the pull stream with
halfway bounce-back (Sec. 4.2 split design) delivers along direction i.  This
test restates both rules on random masks, with inflow and outflow planes, on both
lattices and on grids small enough for the periodic wrap to alias neighbours, and
checks that every entry of every FLUID_BOUNDARY cell has exactly one writer,
which is the cell and population that the gather definition names."""
import numpy as np
import pytest

C = [((i % 3) - 1, (i // 3) % 3 - 1, i // 9 - 1) for i in range(27)]


def _entries(orc, shape, mask, inflow, outflow, q19):
    nx, ny, nz = shape
    N = nx * ny * nz
    _, _, cells, words = orc.classify(mask, inflow, outflow)
    dirs = [i for i in range(27) if not q19 or sum(a * a for a in C[i]) <= 2]

    def xyz(n):
        return n % nx, (n // nx) % ny, n // (nx * ny)

    def idx(x, y, z):
        return (x % nx) + nx * ((y % ny) + ny * (z % nz))

    fb = int(orc.FLUID_BOUNDARY)
    # gather definition: entry (i, k) is population i of x - c_i, or population
    # opp(i) of x itself for a solid link
    want, source = {}, np.zeros(N, bool)
    for k, (n, w) in enumerate(zip(cells.tolist(), words.tolist())):
        if (w >> 27) != fb:
            continue
        x, y, z = xyz(n)
        source[n] = True
        for i in dirs:
            if (w >> i) & 1:
                want[(i, k)] = (n, 26 - i)
            else:
                s = idx(x - C[i][0], y - C[i][1], z - C[i][2])
                source[s] = True
                want[(i, k)] = (s, i)
    assert not mask.ravel()[source].any(), "a source cell is solid"
    lidx = np.full(N, -1, np.int64)
    for k, (n, w) in enumerate(zip(cells.tolist(), words.tolist())):
        if (w >> 27) == fb:
            lidx[n] = k
    # push form: every writer of every entry
    got = {}
    for s in np.nonzero(source)[0].tolist():
        x, y, z = xyz(s)
        for i in dirs:
            k = lidx[idx(x + C[i][0], y + C[i][1], z + C[i][2])]
            if k >= 0:
                got.setdefault((i, int(k)), []).append((s, i))
        k = lidx[s]
        if k >= 0:
            w = int(words[k])
            for i in dirs:
                if (w >> i) & 1:
                    got.setdefault((i, int(k)), []).append((s, 26 - i))
    return want, got


@pytest.mark.parametrize("shape", [(12, 9, 7), (7, 5, 4), (5, 3, 2)])
@pytest.mark.parametrize("q19", [False, True])
def test_every_entry_has_exactly_the_writer_the_gather_names(orc, shape, q19):
    rng = np.random.default_rng(sum(shape) + 7 * q19)
    nx, ny, nz = shape
    for dens in (0.1, 0.3):
        for inflow, outflow in ((False, False), (True, True), (True, False)):
            mask = (rng.random((nz, ny, nx)) < dens).astype(np.uint8)
            want, got = _entries(orc, shape, mask, inflow, outflow, q19)
            assert set(got) == set(want)
            for key, writers in got.items():
                assert writers == [want[key]], (key, writers, want[key])


def test_a_planted_push_mistake_is_caught(orc):
    """Pushing to s - c_i instead of s + c_i (the gather's direction) must fail."""
    shape = (7, 5, 4)
    mask = (np.random.default_rng(3).random((4, 5, 7)) < 0.2).astype(np.uint8)
    want, got = _entries(orc, shape, mask, True, True, False)
    flipped = {}
    for (i, k), writers in got.items():
        flipped.setdefault((26 - i, k), []).extend(writers)
    assert flipped != {key: [v] for key, v in want.items()}
