"""Host logic of bench.py (no GPU needed): the digest that keys the DRAM
traffic record of the dominant kernel ignores comments and whitespace and
changes with the code."""
import bench

SRC = """// a kernel
__global__ void k(int *a, int n) /* launch bounds elsewhere */
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = i;  // fill
}
"""


def test_digest_ignores_comments_and_whitespace():
    d = bench.code_digest([SRC])
    edited = SRC.replace("// fill", "// fill the array with its indexes").replace("    ", "\t")
    edited = "/* header\n   over two lines */\n" + edited + "\n\n// trailing note\n"
    assert bench.code_digest([edited]) == d


def test_digest_follows_the_code():
    d = bench.code_digest([SRC])
    assert bench.code_digest([SRC.replace("a[i] = i", "a[i] = 2 * i")]) != d
    assert bench.code_digest([SRC.replace("i < n", "i <= n")]) != d
    assert bench.code_digest([SRC, SRC]) != d  # more code, another digest


def test_source_hash_is_stable():
    assert bench.source_hash() == bench.source_hash()
    assert len(bench.source_hash()) == 16
