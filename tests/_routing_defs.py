"""Routing tables rebuilt from their definitions with numpy (test helper):
the internal order, the CSR sorted by (destination partition, delay, target,
weight), one level-2 entry per destination-partition run (length, partition,
relay class, delay-1 count), one level-1 entry per destination-VN run, and the
exchange pairs with their worst-case capacities (Sec. IV.B: level 1 to the
destination VN's relay, level 2 from the relay to the partition)."""
import numpy as np

L2_DTYPE = np.dtype([("off", "<u8"), ("len", "<u4"), ("q", "<u2"), ("cls", "u1"), ("pad", "u1")])


def check_tables(rt, g, part, P, n_vn):
    """Assert that every table rt exports (host- or device-built) follows
    from the network g and the mapping part (per_vn relays, VNs of P / n_vn
    partitions)."""
    s = P // n_vn
    vn = rt.export("vn_of_part")
    # internal partition order: by (VN, label); neurons partition-major, ascending ids
    ip_of = np.empty(P, np.int64)
    fill = np.zeros(n_vn, np.int64)
    for p in range(P):
        ip_of[p] = vn[p] * s + fill[vn[p]]
        fill[vn[p]] += 1
    inv = rt.export("perm_inv").astype(np.int64)
    fwd = rt.export("perm_fwd").astype(np.int64)
    assert np.array_equal(fwd[inv], np.arange(g.M))
    assert np.array_equal(inv, np.lexsort((np.arange(g.M), ip_of[part])))
    src_part = rt.export("src_part").astype(np.int64)
    assert np.array_equal(src_part, ip_of[part[inv]])
    assert np.array_equal(rt.export("v0"), g.v0[inv])
    deg = np.diff(g.syn_ptr)
    csr = rt.export("csr")
    assert np.array_equal(np.diff(csr), deg[inv])
    td = rt.export("syn_td").astype(np.int64)
    w = rt.export("syn_w")
    l1p = rt.export("l1_ptr").astype(np.int64)
    l1vn = rt.export("l1_vn").astype(np.int64)
    l1l2 = rt.export("l1_l2").astype(np.int64)
    l2 = rt.export("l2").view(L2_DTYPE)
    l1pair = rt.export("l1_pair").astype(np.int64)
    l2pair = rt.export("l2_pair").astype(np.int64)
    bptr, bdst, bcap = rt.export("bpair_ptr"), rt.export("bpair_dst"), rt.export("bpair_cap")
    iptr, idst, icap = rt.export("ipair_ptr"), rt.export("ipair_dst"), rt.export("ipair_cap")
    assert l1l2[-1] == len(l2) and l1p[-1] == len(l1vn)
    icnt = np.zeros((P, P), np.int64)
    bcnt = np.zeros((P, n_vn), np.int64)
    for k in range(g.M):
        i = inv[k]
        ps, hs = src_part[k], src_part[k] // s
        e = slice(g.syn_ptr[i], g.syn_ptr[i + 1])
        tq = ip_of[part[g.tgt[e].astype(np.int64)]]
        want = sorted(zip(tq.tolist(), (g.d[e].astype(np.int64) - 1).tolist(),
                          fwd[g.tgt[e].astype(np.int64)].tolist(), g.w[e].astype(np.uint16).tolist()))
        o = slice(csr[k], csr[k + 1])
        got_t, got_d = td[o] & ((1 << 28) - 1), td[o] >> 28
        got = list(zip(ip_of[part[inv[got_t]]].tolist(), got_d.tolist(), got_t.tolist(),
                       w[o].astype(np.uint16).tolist()))
        assert got == want
        runs = [(q, sum(1 for x in want if x[0] == q)) for q in sorted(set(x[0] for x in want))]
        f0, f1 = l1l2[l1p[k]], l1l2[l1p[k + 1]]
        assert f1 - f0 == len(runs)
        start = csr[k]
        for (q, n), f in zip(runs, range(f0, f1)):
            ent = l2[f]
            assert ent["off"] & ((1 << 40) - 1) == start and ent["len"] == n and ent["q"] == q
            assert ent["off"] >> 40 == sum(1 for x in want if x[0] == q and x[1] == 0)
            gq = q // s
            cls = (0 if q == ps else 1) if gq == hs else (2 if q == gq * s + (hs - gq) % s else 3)
            assert ent["cls"] == cls
            pid = l2pair[f]
            assert iptr[ps] <= pid < iptr[ps + 1] and idst[pid] == q
            icnt[ps, q] += 1
            start += n
        vns = sorted(set(q // s for q, _ in runs))
        assert list(l1vn[l1p[k]:l1p[k + 1]]) == vns
        for e1, gg in zip(range(l1p[k], l1p[k + 1]), vns):
            first = next(j for j, (q, _) in enumerate(runs) if q // s == gg)
            assert l1l2[e1] == f0 + first
            pid = l1pair[e1]
            assert bptr[ps] <= pid < bptr[ps + 1] and bdst[pid] == gg
            bcnt[ps, gg] += 1
    # pairs: exactly those carrying entries, each with its worst case, by source then destination
    assert [(ps, q) for ps in range(P) for q in range(P) if icnt[ps, q]] == \
        [(ps, int(idst[x])) for ps in range(P) for x in range(iptr[ps], iptr[ps + 1])]
    assert list(icap) == [int(icnt[ps, idst[x]]) for ps in range(P) for x in range(iptr[ps], iptr[ps + 1])]
    assert list(bcap) == [int(bcnt[ps, bdst[x]]) for ps in range(P) for x in range(bptr[ps], bptr[ps + 1])]
    assert np.array_equal(rt.export("inbox_cap"), icnt.sum(0))
    assert np.array_equal(rt.export("bucket_cap"), bcnt.sum(0))
