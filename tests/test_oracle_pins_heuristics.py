"""Pins of three oracle functions to values fixed outside the oracle (no GPU).

* Philox4x32 at 10 rounds against the known-answer vectors published with the
  generator (Salmon, Moraes, Dror, Shaw, SC'11; the Random123 distribution's
  test vectors): zero key and counter, all-ones, and the pi-digit case.
* The heuristic default policy of Rock Sample (Sec. IV-A; the reading:
  sample a believed-good rock underfoot, else step toward the nearest
  believed-good unsampled rock by Manhattan distance with the lowest index on
  ties and the x-move before the y-move, else go east) on hand-worked maps.
  Each expected action is derived by hand from that rule.
* The upper-bound heuristic u (Eq. ub's u0 per scenario; the reading: every
  good rock at its nearest robot's Manhattan distance, 10 * gamma^d, plus each
  robot's exit 10 * gamma^(n-1-x)) as closed-form sums of powers of gamma.

Each test fails if its function is mutated in a plausible way: the round count,
ties broken toward the highest index, y-move first, counters of 0 believed good,
sampled rocks kept as targets, gamma^(d+1) for gamma^d, a dropped exit term, or
the multi-robot minimum replaced by the first robot.
"""
import numpy as np

import oracle
from paper_1802_06215_b300 import inputs as I

N, E, S, W, SAMPLE = 0, 1, 2, 3, 4


# ---------------------------------------------------------------- Philox-10 --

PHILOX10_KAT = [
    # counter (4 words), key (2 words), output (4 words)
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


def test_philox10_known_answer_vectors():
    for ctr, key, want in PHILOX10_KAT:
        got = oracle.philox(ctr, key[0], key[1], 10)
        assert [int(x) for x in got] == list(want)


def test_philox10_kat_rejects_other_round_counts():
    """The vectors are specific to 10 rounds: 7, 9 and 11 rounds miss them."""
    ctr, key, want = PHILOX10_KAT[2]
    for r in (7, 9, 11):
        assert [int(x) for x in oracle.philox(ctr, key[0], key[1], r)] != list(want)


# ----------------------------------------------------------- default policy --

def _cfg(rocks, n=7, robots=1):
    cells = np.array([x | (y << 8) for x, y in rocks], np.int32)
    return I.Config(kind=I.GRID if robots == 1 else I.MULTIGRID, n=n, m=len(rocks), K=8, D=10, seed=3,
                    rock_cells=cells)


def _block(robots, sampled=0, good=0):
    b = np.zeros((5, 1), np.uint32)
    for r, (x, y) in enumerate(robots):
        b[r, 0] = x | (y << 8)
    b[2, 0], b[3, 0], b[4, 0] = good, sampled, 0
    return b


def _hist(counters):
    h = np.zeros((1, 32), np.int8)
    h[0, :len(counters)] = counters
    return h


def _act(rocks, robot, counters, sampled=0):
    cfg = _cfg(rocks)
    return int(oracle.Model(cfg).policy(_block([robot], sampled), _hist(counters))[0])


def test_policy_no_candidate_goes_east():
    rocks = [(4, 3), (0, 0)]
    assert _act(rocks, (2, 3), [0, 0]) == E          # counters of 0 are not believed good
    assert _act(rocks, (2, 3), [-2, -1]) == E        # believed bad
    assert _act(rocks, (2, 3), [3, 2], sampled=0b11) == E  # all sampled


def test_policy_equal_distances_lowest_index_wins():
    # robot (2,3); rock 0 west at distance 2, rock 1 east at distance 2
    assert _act([(0, 3), (4, 3)], (2, 3), [1, 1]) == W
    # the same rocks listed the other way round
    assert _act([(4, 3), (0, 3)], (2, 3), [1, 1]) == E
    # three-way tie at distance 3: rock 0 north, rock 1 south, rock 2 east -> rock 0
    assert _act([(2, 6), (2, 0), (5, 3)], (2, 3), [1, 1, 1]) == N
    # the tie goes to the lowest index among the believed-good rocks only
    assert _act([(2, 6), (2, 0), (5, 3)], (2, 3), [0, 2, 1]) == S


def test_policy_nearest_wins_over_index():
    # rock 0 at distance 4 (north-east), rock 1 at distance 1 (south)
    assert _act([(4, 5), (2, 2)], (2, 3), [1, 1]) == S


def test_policy_x_move_before_y_move():
    # diagonal targets: the x-move comes first in every quadrant
    assert _act([(4, 5)], (2, 3), [1]) == E
    assert _act([(0, 5)], (2, 3), [1]) == W
    assert _act([(5, 0)], (2, 3), [1]) == E
    assert _act([(1, 1)], (2, 3), [1]) == W
    # same column: the y-move, N is y+1
    assert _act([(2, 6)], (2, 3), [1]) == N
    assert _act([(2, 0)], (2, 3), [1]) == S


def test_policy_skips_sampled_and_unbelieved_nearer_rocks():
    rocks = [(3, 3), (2, 6), (0, 3)]    # distances 1, 3, 2 from (2,3)
    # nearest rock 0 already sampled -> rock 2 (distance 2, west)
    assert _act(rocks, (2, 3), [2, 1, 1], sampled=0b001) == W
    # nearest rock 0 with counter 0 -> rock 2
    assert _act(rocks, (2, 3), [0, 1, 1]) == W
    # rocks 0 and 2 not believed good -> rock 1 north
    assert _act(rocks, (2, 3), [-1, 1, 0]) == N


def test_policy_samples_rock_underfoot_among_others():
    rocks = [(1, 3), (2, 3), (3, 3)]
    assert _act(rocks, (2, 3), [1, 1, 1]) == SAMPLE
    # the rock underfoot is believed bad: walk to the nearest other (rock 0 wins the tie)
    assert _act(rocks, (2, 3), [1, -1, 1]) == W
    # the rock underfoot was sampled
    assert _act(rocks, (2, 3), [0, 5, 1], sampled=0b010) == E


def test_policy_two_robots_joint_action():
    rocks = [(4, 3), (1, 1)]
    cfg = _cfg(rocks, robots=2)
    per = 5 + len(rocks)
    b = _block([(2, 3), (1, 4)])
    # robot 0 -> rock 0 (distance 2, E); robot 1 -> rock 1 (distance 3, same column, S)
    a = int(oracle.Model(cfg).policy(b, _hist([1, 1]))[0])
    assert a == E * per + S
    # robot 1 stands on rock 1
    b = _block([(2, 3), (1, 1)])
    a = int(oracle.Model(cfg).policy(b, _hist([1, 1]))[0])
    assert a == E * per + SAMPLE


# ---------------------------------------------------------------- u bound --

G = float(np.float32(0.95))   # the model's FP32 gamma, its powers taken in FP64


def _upper(rocks, robots, good, n=7, fp64=True):
    cfg = _cfg(rocks, n=n, robots=len(robots))
    u, _ = oracle.Model(cfg, fp64=fp64).bounds(_block(robots, good=good))
    return float(u[0])


def test_upper_one_good_rock():
    # robot (2,3), rock (4,3): d = 2; exit from x = 2 on n = 7: 4 steps
    assert abs(_upper([(4, 3)], [(2, 3)], 0b1) - (10 * G**2 + 10 * G**4)) < 1e-12
    # rock (0,6): d = 2 + 3 = 5
    assert abs(_upper([(0, 6)], [(2, 3)], 0b1) - (10 * G**5 + 10 * G**4)) < 1e-12


def test_upper_two_rocks_and_bad_rock():
    rocks = [(4, 3), (0, 6), (6, 0)]
    want = 10 * G**2 + 10 * G**5 + 10 * G**4          # rock 2 (d = 7) is bad
    assert abs(_upper(rocks, [(2, 3)], 0b011) - want) < 1e-12
    want_all = want + 10 * G**7
    assert abs(_upper(rocks, [(2, 3)], 0b111) - want_all) < 1e-12


def test_upper_rock_underfoot_and_east_edge():
    # a good rock underfoot counts 10 * gamma^0; at x = n-1 the exit term is 10
    assert abs(_upper([(6, 2)], [(6, 2)], 0b1) - 20.0) < 1e-12
    assert abs(_upper([(0, 0)], [(6, 2)], 0b0) - 10.0) < 1e-12


def test_upper_two_robots_minimum_distance():
    rocks = [(4, 3), (0, 0)]
    # robot 0 (2,3): d = 2 and 5; robot 1 (5,3): d = 1 and 8; exits 4 and 1 steps
    want = 10 * G**1 + 10 * G**5 + 10 * G**4 + 10 * G**1
    assert abs(_upper(rocks, [(2, 3), (5, 3)], 0b11) - want) < 1e-12


def test_upper_fp32_matches_closed_form():
    got = _upper([(4, 3), (0, 6)], [(2, 3)], 0b11, fp64=False)
    want = 10 * G**2 + 10 * G**5 + 10 * G**4
    assert abs(got - want) < 1e-5 * want


def test_scenario_streams_use_ten_rounds():
    """phi_t of a scenario is the 10-round block at counter (scenario, depth,
    purpose<<24 | element, planning step) under key (seed low, seed high), so
    the known-answer vectors above pin every stream the models draw."""
    seed = 0x0123456789ABCDEF
    for scen, depth, purpose, elem, step in [(0, 0, 0, 0, 0), (7, 3, 2, 1, 5), (499, 89, 3, 12, 99)]:
        got = oracle.scenario_random(seed, scen, depth, purpose, elem, step)
        ctr = (scen, depth, (purpose << 24) | elem, step)
        want = oracle.philox(ctr, seed & 0xFFFFFFFF, seed >> 32, 10)
        assert np.array_equal(got, want)
