"""Index model of the phased chain schedule of the cluster-resident solve
(host-side restatement of the launch and segment arithmetic, checked before
any GPU run): in launch p of nch, cluster slot s takes chain
c = s if s < p else s + 1 and contour steps (m_begin, m_end] of its segment
seg = p if p < c else p - 1, with segment bounds seg * N_s // (nch - 1).
Every chain must run every step exactly once, in order, resume where its
previous launch stopped, and never share a launch with itself."""
import pytest


def chain_of(slot, skip, nseg):
    return slot if (nseg == 0 or slot < skip) else slot + 1


def segment(chain, skip, nseg, ns):
    if nseg == 0:
        return 0, ns
    seg = skip if skip < chain else skip - 1
    return seg * ns // nseg, (seg + 1) * ns // nseg


CASES = [(nch, ns) for nch in (2, 4, 6, 8, 16, 20) for ns in (nch - 1, 17, 64, 128, 512) if ns >= nch - 1]


@pytest.mark.parametrize("nch,ns", CASES)
def test_every_chain_runs_every_step_once_in_order(nch, ns):
    # N_s >= nch - 1: the launcher takes the phased schedule only then
    nseg = nch - 1
    done = {c: 0 for c in range(nch)}
    for p in range(nch):  # launch p
        seen = set()
        for slot in range(nseg):
            c = chain_of(slot, p, nseg)
            assert 0 <= c < nch and c != p and c not in seen
            seen.add(c)
            m0, m1 = segment(c, p, nseg, ns)
            assert m0 == done[c]  # resumes from the state its last launch stored
            assert 1 <= m1 - m0 and m1 <= ns
            done[c] = m1
        assert seen == set(range(nch)) - {p}
    assert all(v == ns for v in done.values())


def test_single_launch_is_the_whole_chain():
    for slot in range(8):
        assert chain_of(slot, 0, 0) == slot
        assert segment(slot, 0, 0, 64) == (0, 64)


def test_phase_lengths_on_the_benchmark_batch():
    # 4 runs, N_s = 64: segments of 9 steps and a last one of 10, which runs
    # in two launches (chain 7 in launch 6, the others in launch 7); the
    # launches together take 74 step lengths against 64 for one run alone
    nch, ns = 8, 64
    lengths = []
    for p in range(nch):
        spans = [segment(chain_of(s, p, nch - 1), p, nch - 1, ns) for s in range(nch - 1)]
        lengths.append(max(m1 - m0 for m0, m1 in spans))
    assert lengths == [9] * 6 + [10, 10] and sum(lengths) == 74
