"""The operation counter of oracle/op_count.py, pinned on expressions whose
cost is known by hand, and the per-cell work of the quantum model it derives
from the oracle's expression, set beside the counts the roofline of the bench
kernel uses (the kernel's own packed-instruction counts)."""


def _op_count():
    from oracle import op_count
    return op_count


def _bench_constants():
    import bench
    return bench


def test_counter_on_hand_counted_expressions():
    oc = _op_count()
    g = oc.Graph()
    x, y, z = (oc.V(g, g.var(n)) for n in "xyz")
    a = oc.V(g, g.inv("a"))
    # x y + z: one FMA
    assert oc.count([(x * y + z).n])["fma_pipe"] == 1
    # (x y) + (x y): the product once (common subexpression) and one add;
    # the product has two uses, so it is not fused -- two operations
    p = x * y
    assert oc.count([(p + p).n])["fma_pipe"] == 2
    # x / y: a reciprocal and a product; x / a (a invariant): one product
    c1 = oc.count([(x / y).n])
    assert c1["mufu_slots"] == 1.0 and c1["fma_pipe"] == 1
    assert oc.count([(x / a).n]) == {"adds": 0, "muls": 1, "fused": 0, "fma_pipe": 1,
                                     "mufu_slots": 0.0}
    # log(x) and x**(-2/3): lg2 (+ ex2 at half a slot) and a product each
    assert oc.count([x.log().n])["mufu_slots"] == 1.0
    assert oc.count([x.powf(-2.0 / 3.0).n])["mufu_slots"] == 1.5
    # invariant subtrees cost nothing: (a * a + a) * x is one product
    assert oc.count([((a * a + a) * x).n])["fma_pipe"] == 1
    # a product used twice is not fused: x y + z and x y - x
    q = x * y
    c2 = oc.count([(q + z).n, (q - x).n])
    assert c2["fma_pipe"] == 3


def test_quantum_cell_counts_against_the_bench_constants():
    oc = _op_count()
    cnt = oc.cell_counts()
    print("oracle expression, one phase cell:", cnt)
    b = _bench_constants()
    # the counts the bench's roofline divides by (the FP32 kernel's own packed
    # instructions) are at most the oracle expression's: the kernel reaches
    # the same quantities with fewer operations, so its roofline fraction is
    # the lower of the two
    assert cnt["fma_pipe"] == b.ORACLE_CELL_FMA_OPS
    assert cnt["mufu_slots"] == b.ORACLE_CELL_MUFU_SLOTS
    assert b.QFP_FMA_OPS_PER_STEP <= cnt["fma_pipe"]
    assert b.QFP_MUFU_SLOTS_PER_STEP <= cnt["mufu_slots"]
