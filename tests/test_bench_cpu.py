"""bench.py's roofline arithmetic on the CPU: the algorithmic work per chunk
that the bench line divides by the kernel time, checked against the cost
model's closed forms (one CIOS Montgomery product = 2 s^2 + s MACs over s
limbs; one full-d decryption at the fixed w = 5 window count = (n - 1)
squarings + n/6 multiplies + 16 table entries + 2 conversions)."""
import pytest

import bench


@pytest.mark.parametrize("nbits,macs", [(1024, 2080), (2048, 8256), (3072, 18528), (4096, 32896)])
def test_montmul_macs(nbits, macs):
    s = nbits // 32
    assert bench.macs_per_montmul(nbits) == macs == 2 * s * s + s


def test_full_d_count_at_2048_bits():
    n = 2048
    assert bench.algorithmic_montmuls(n) == pytest.approx(2047 + 2048 / 6 + 18)
    assert bench.algorithmic_montmuls(n) == pytest.approx(2406.33, abs=0.01)
    assert bench.algorithmic_montmuls(n) * bench.macs_per_montmul(n) == pytest.approx(1.987e7, rel=1e-3)


def test_crt_count_and_prime_scaling():
    # two primes at 2048 bits: two 1024-bit exponentiations, 3 input products each, 2 recombination products
    two = bench.algorithmic_crt_macs(2048, 2)
    assert two == pytest.approx(2 * (bench.algorithmic_montmuls(1024) + 3) * 2080 + 2 * 8256)
    assert two == pytest.approx(5.07e6, rel=1e-3)
    # b primes of n/b bits: each exponentiation costs ~ (n/b)^3, so the total falls ~ b^2 / 4 against two primes
    for n, b in ((2048, 4), (3072, 3), (4096, 4), (8192, 4)):
        ratio = bench.algorithmic_crt_macs(n, 2) / bench.algorithmic_crt_macs(n, b)
        assert 0.8 * b * b / 4 < ratio < 1.05 * b * b / 4, (n, b, ratio)


def test_int32_roofline_recomputes_from_its_inputs():
    # The headline fraction: 2 INT32 multiply-add halves per MAC over the measured mad.lo rate.  With the
    # 1 MiB / K = 8 / 2048-bit workload (4,113 chunks), a 17.63 ms decryption and 63.99 mad.lo per clock per
    # SM on 152 SMs at 2070 MHz, the figure is 9.27 of 20.13 TOP/s.
    macs = bench.algorithmic_montmuls(2048) * bench.macs_per_montmul(2048) * 4113
    achieved = bench.int32_ops_per_s(macs, 17.63) / 1e12
    peak = bench.int32_peak_tops(63.99, 152, 2070.0)
    assert achieved == pytest.approx(9.27, abs=0.01)
    assert peak == pytest.approx(20.13, abs=0.01)
    assert achieved / peak == pytest.approx(0.46, abs=0.005)


def test_issue_slots_follow_the_current_kernel_sources():
    # The stored counters are reported only for the kernel sources they were captured on, and the
    # instructions per MAC come from the capture's warp instruction count: 1.007e10 warp instructions
    # for 8.17e10 algorithmic MACs are 3.94 thread instructions per MAC.
    macs = bench.algorithmic_montmuls(2048) * bench.macs_per_montmul(2048) * 4113
    got = bench.issue_slots({"issue_active_pct": 51.06, "warps_active_per_sm": 6.91, "alu_pipe_pct": 56.93,
                             "fmaheavy_pipe_pct": 61.13, "warp_instructions": 10071705714}, macs)
    assert got["thread_instructions_per_mac"] == pytest.approx(3.94, abs=0.01)
    assert bench.issue_slots({}, macs) is None
    for counters in bench.COUNTERS_MEASURED.values():
        assert set(counters) >= {"traffic", "issue_active_pct", "warp_instructions"}


def test_counter_digest_ignores_comments_only():
    a = "int f(int x) {  // add one\n  return x + 1; /* plain */ }\n"
    b = "int f(int x) {\n  // adds 1 to x\n  return x + 1;\n}\n"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_digest([a]) == bench.code_digest([b])
    assert bench.code_digest([a]) != bench.code_digest([c])
