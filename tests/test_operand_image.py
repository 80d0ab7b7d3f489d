"""The tensor-core operand images (host-side set-up of the contraction) decoded on the CPU from
the canonical no-swizzle K-major layout as include/coffee_diag.h defines it: every image holds
the reference tensor T^T (rows = element-matrix entries, columns = K) to the accuracy of its
precision split (TF32 one part, TF32X3 and BF16 two, BF16X3 three), zero padding elsewhere;
the stiffness columns of HELMHOLTZ and ADVDIFF are re-expressed for the edge factors
c_ij = |det J| grad(lambda_i).grad(lambda_j), and the Burgers images use exact integer columns
where the paper's tensors allow them. No GPU needed."""
import ctypes
import math

import numpy as np
import pytest

import paper_1407_0904_gb300 as coffee

TRI, TET = coffee.TRIANGLE, coffee.TETRAHEDRON
TPARTS = {coffee.TF32: 1, coffee.TF32X3: 2, coffee.BF16: 2, coffee.BF16X3: 3}
TF32 = {coffee.TF32X3: True, coffee.TF32: True, coffee.BF16X3: False, coffee.BF16: False}


def image(form, k, cell, prec):
    L = coffee.lib()
    L.coffee_table_image.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 3
    n = ctypes.c_int64()
    meta = (ctypes.c_int64 * 8)()
    rc = L.coffee_table_image(form, k, cell, prec, None, ctypes.byref(n), meta)
    if rc == -2:
        return None
    assert rc == 0, L.coffee_last_error()
    img = np.zeros(n.value, dtype=np.uint8)
    assert L.coffee_table_image(form, k, cell, prec, img.ctypes.data, ctypes.byref(n), None) == 0
    return img, list(meta)


def decode(part, kbytes, tf32):
    """One 128-row part -> float32 [128, kbytes / elem] from its canonical layout."""
    r = np.arange(128)[:, None]
    kb = np.arange(kbytes)[None, :]
    off = (r // 8) * 8 * kbytes + (kb // 16) * 128 + (r % 8) * 16 + kb % 16
    raw = np.ascontiguousarray(part[off])                      # logical (row, byte) order
    if tf32:
        bits = raw.view(np.uint32)
        assert np.all(bits & 0x1FFF == 0)                      # tf32: 10 stored mantissa bits
        return bits.view(np.float32)
    return (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32)


def operand(img, meta, tf32, aparts):
    """(first part, sum of the remaining parts) of the A operand, each [mtiles*128, kelems]."""
    mtiles, kbytes = meta[0], meta[1]
    tile = 128 * kbytes
    hi, rest = [], []
    for m in range(mtiles):
        base = m * aparts * tile
        parts = [decode(img[base + q * tile:base + (q + 1) * tile], kbytes, tf32).astype(np.float64)
                 for q in range(aparts)]
        hi.append(parts[0])
        rest.append(sum(parts[1:]) if aparts > 1 else np.zeros_like(parts[0]))
    return np.vstack(hi), np.vstack(rest)


def edge_basis(T, r0, d):
    """Rows r0.. r0+P-1 of T (stiffness pairs a <= b of reference directions) re-expressed for the
    edge factors c_ij, i < j over the d+1 vertices: H_ab = c_(a+1)(b+1) for a != b and
    H_aa = -sum_(j != a+1) c_(a+1)j, since the barycentric gradients sum to zero."""
    pairs = [(a, b) for a in range(d) for b in range(a, d)]
    row = {p: r0 + i for i, p in enumerate(pairs)}
    out = T.copy()
    e = r0
    for i in range(d + 1):
        for j in range(i + 1, d + 1):
            if i == 0:
                out[e] = -T[row[(j - 1, j - 1)]]
            else:
                out[e] = T[row[(i - 1, j - 1)]] - T[row[(i - 1, i - 1)]] - T[row[(j - 1, j - 1)]]
            e += 1
    return out


CASES = [(f, c, k, p) for f in (coffee.MASS, coffee.HELMHOLTZ, coffee.ADVDIFF) for c in (TRI, TET)
         for k in (1, 2, 3, 4) for p in (coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16)]


@pytest.mark.parametrize("form,cell,k,prec", CASES)
def test_simplex_image_holds_the_reference_tensor(form, cell, k, prec):
    got = image(form, k, cell, prec)
    if got is None:
        pytest.skip("no tensor-core kernel for this combination")
    img, meta = got
    mtiles, kbytes, kelems, K, parts = meta[:5]
    tf32 = TF32[prec]
    T = coffee.reference_tensor(form, k, cell)                 # [K, N]
    N = T.shape[1]
    d = 2 + cell
    P = d * (d + 1) // 2
    if form == coffee.HELMHOLTZ:
        T = edge_basis(T, 1, d)
    elif form == coffee.ADVDIFF:
        for v in range(d + 1):
            T = edge_basis(T, v * P, d)
    assert K == T.shape[0] and mtiles == math.ceil(N / 128) and parts == TPARTS[prec]
    assert kelems * (4 if tf32 else 2) == kbytes and kbytes % 32 == 0 and kelems >= K
    assert len(img) == mtiles * parts * 128 * kbytes
    hi, lo = operand(img, meta, tf32, parts)
    ref = np.zeros_like(hi)
    ref[:N, :K] = T.T
    # padding rows and columns are zero
    assert not hi[N:].any() and not hi[:, K:].any() and not lo[N:].any() and not lo[:, K:].any()
    u = 2.0 ** -11 if tf32 else 2.0 ** -8                      # unit roundoff: 11 or 8 significant bits
    bound = u ** parts * 1.01 * np.abs(ref) + 1e-300           # each part rounds what the previous left
    assert np.all(np.abs(hi + lo - ref) <= bound)
    assert np.all(np.abs(hi - ref) <= u * 1.01 * np.abs(ref) + 1e-300)


@pytest.mark.parametrize("cell,k", [(TRI, 1), (TRI, 2), (TRI, 3), (TET, 1), (TET, 2)])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3])
def test_burgers_image_exact_integer_columns(cell, k, prec):
    """P1-P2 on triangles and tetrahedra: every A column is an integer vector times a float scale
    (one part, one MMA pass per part of the factors); triangles P3 keep the split image. The
    columns are T1, then the T2 and T3 rows of coffee_reference_tensor(BURGERS_JAC) after the
    off-diagonal K-steps."""
    got = image(coffee.BURGERS_JAC, k, cell, prec)
    if got is None:
        pytest.skip("no tensor-core kernel for this combination")
    img, meta = got
    mtiles, kbytes, kelems, K, parts, aexact, ksteps_off, scale_off = meta
    tf32 = TF32[prec]
    assert aexact == (1 if k <= 2 else 0) and parts == (1 if aexact else TPARTS[prec])
    T = coffee.reference_tensor(coffee.BURGERS_JAC, k, cell)
    d = 2 + cell
    ns = coffee.nnodes(cell, k)
    nb = ns * ns
    K1, P = ns * d, d * (d + 1) // 2
    KA1 = ksteps_off * (8 if tf32 else 16)
    assert KA1 >= K1 and K == KA1 + K1 + P == T.shape[0] + (KA1 - K1)
    hi, lo = operand(img, meta, tf32, parts)
    A = hi + lo
    if aexact:
        ints = hi
        assert np.all(ints == np.round(ints)) and not lo.any()
        odd = np.abs(ints).astype(np.int64)
        while np.any((odd > 0) & (odd % 2 == 0)):
            odd = np.where((odd > 0) & (odd % 2 == 0), odd // 2, odd)
        assert odd.max() < (2048 if tf32 else 256)
        scales = np.frombuffer(img[scale_off:scale_off + 4 * kelems].tobytes(), dtype=np.float32)
        assert np.all(np.isfinite(scales)) and np.all(scales > 0)
        A = ints * scales[None, :].astype(np.float64)
    trow = [kk if kk < K1 else ns * d + kk - KA1 if KA1 <= kk < KA1 + K1
            else 2 * ns * d + kk - KA1 - K1 if KA1 + K1 <= kk < KA1 + K1 + P else -1 for kk in range(kelems)]
    for kk, tr in enumerate(trow):
        col = np.zeros(mtiles * 128)
        if tr >= 0:
            col[:nb] = T[tr]
        scale = max(np.abs(col).max(), 1e-300)
        tol = 2.0 ** -23 if aexact else ((2.0 ** -22) if tf32 else 2.0 ** -24) * 1.01
        assert np.abs(A[:, kk] - col).max() <= tol * scale, (kk, tr)


@pytest.mark.parametrize("form", [coffee.MASS, coffee.HELMHOLTZ, coffee.ADVDIFF])
@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3])
def test_prism_image_holds_the_per_point_tensors_of_the_oracles_basis(form, k, prec):
    """Prisms: K-chunks of 64 bytes per row (all 128-output slices, their parts in order), then
    the rule's points and weights as float4. The rule is the oracle's (as a set of points), and
    column q*KQ + c holds, at point q, phi_i phi_j (MASS, HELMHOLTZ c = 0), the symmetric
    derivative pairs (HELMHOLTZ c = 1..6, ADVDIFF c = 0..5) and phi_i d_a phi_j (ADVDIFF
    c = 6..8), evaluated here with the oracle's own prism basis: an independent check of the
    GPU side's prism tabulation and of the streamed layout. The last chunk holds the
    weight-summed tensors sum_q w_q T[q*KQ+c] in its first KQ columns (the centre factors'
    contraction)."""
    import oracle
    img, meta = image(form, k, coffee.PRISM, prec)
    mtiles, kbytes, kelems, K, parts, _, KQ, _ = meta
    tf32 = TF32[prec]
    kc = kbytes // (4 if tf32 else 2)
    nkc = kelems // kc
    n = oracle.prism_ndof(k)
    N, Q = n * n, (k + 2) ** 3
    assert KQ == {coffee.MASS: 1, coffee.HELMHOLTZ: 7, coffee.ADVDIFF: 9}[form] and K == Q * KQ
    assert mtiles == math.ceil(N / 128) and parts == TPARTS[prec] and nkc == math.ceil(K / kc) + 1
    tb = 128 * kbytes
    a_chunk = mtiles * parts * tb
    assert len(img) == nkc * a_chunk + 16 * Q
    cols = []
    for c in range(nkc):
        rows = []
        for m in range(mtiles):
            base = c * a_chunk + m * parts * tb
            rows.append(sum(decode(img[base + q * tb:base + (q + 1) * tb], kbytes, tf32).astype(np.float64)
                            for q in range(parts)))
        cols.append(np.vstack(rows))
    A = np.hstack(cols[:-1])                                   # [mtiles*128, (nkc-1)*kc]
    Abar = cols[-1]
    assert not A[N:].any() and not A[:, K:].any() and not Abar[N:].any() and not Abar[:, KQ:].any()
    table = np.frombuffer(img[nkc * a_chunk:].tobytes(), dtype=np.float32).reshape(Q, 4).astype(np.float64)
    pts, wts = table[:, :3], table[:, 3]
    opts, owts = oracle.prism_rule(k)
    assert len(owts) == Q
    near = np.argmin(((pts[:, None, :] - opts[None, :, :]) ** 2).sum(-1), axis=1)
    assert len(np.unique(near)) == Q
    assert np.abs(pts - opts[near]).max() < 1e-6 and np.abs(wts - owts[near]).max() < 1e-6 * owts.max()
    phi, dphi = oracle.prism_basis(k, pts)
    pairs = [(a, b) for a in range(3) for b in range(a, 3)]
    tol = 1e-5 if tf32 else 5e-5
    wsum = [0.0] * KQ
    for q in range(Q):
        want = []
        if KQ != 9:
            want.append(np.outer(phi[q], phi[q]))
        if KQ >= 7:
            for a, b in pairs:
                v = np.outer(dphi[q, :, a], dphi[q, :, b])
                if a != b:
                    v = v + np.outer(dphi[q, :, b], dphi[q, :, a])
                want.append(v)
        if KQ == 9:
            want += [np.outer(phi[q], dphi[q, :, a]) for a in range(3)]
        for c, w in enumerate(want):
            got = A[:N, q * KQ + c]
            scale = max(np.abs(w).max(), 1e-12)
            assert np.abs(got - w.ravel()).max() <= tol * scale, (q, c)
            wsum[c] = wsum[c] + owts[near[q]] * w.ravel()
    for c in range(KQ):
        assert np.abs(Abar[:N, c] - wsum[c]).max() <= tol * np.abs(wsum[c]).max(), c


@pytest.mark.parametrize("cell,k", [(TRI, 1), (TRI, 2), (TRI, 3), (TRI, 4), (TET, 1), (TET, 2)])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16])
def test_residual_image_holds_t2_and_t3(cell, k, prec):
    """The residual contracts only the T2 and T3 tensors of the Jacobian: its image holds
    [T2 | T3]^T (columns = the d ns T2 rows of the Burgers reference tensor, then its P T3 rows),
    split into the precision's parts of T, zero in the padding rows and columns."""
    got = image(coffee.BURGERS_RESIDUAL, k, cell, prec)
    if got is None:
        pytest.skip("no tensor-core kernel for this combination")
    img, meta = got
    mtiles, kbytes, kelems, K, parts, aexact, _, _ = meta
    d, ns = 2 + cell, coffee.nnodes(cell, k)
    nb, K1, P = ns * ns, ns * d, d * (d + 1) // 2
    assert mtiles == (nb + 127) // 128 and aexact == 0 and parts == TPARTS[prec] and K == K1 + P
    tf32 = TF32[prec]
    assert kelems * (4 if tf32 else 2) == kbytes and kelems % (8 if tf32 else 16) == 0 and kelems >= K
    hi, rest = operand(img, meta, tf32, parts)
    A = hi + rest
    T = coffee.reference_tensor(coffee.BURGERS_JAC, k, cell).reshape(-1, nb)
    want = np.zeros((128 * mtiles, kelems))
    want[:nb, :K] = T[K1:K1 + K].T
    tol = {coffee.TF32X3: 2.0 ** -21, coffee.BF16X3: 2.0 ** -23, coffee.TF32: 2.0 ** -10,
           coffee.BF16: 2.0 ** -15}[prec]
    assert np.all(A[nb:] == 0) and np.all(A[:, K:] == 0)
    assert np.abs(A - want).max() <= tol * np.abs(T).max()


@pytest.mark.parametrize("cell,k", [(TET, 3), (TET, 4), (TRI, 4)])
@pytest.mark.parametrize("prec", [coffee.TF32X3, coffee.BF16X3, coffee.TF32, coffee.BF16])
def test_burgers_streamed_image_chunks(cell, k, prec):
    """Shapes whose operands do not fit in shared memory (tetrahedra P3-P4, triangles P4 in the
    split precisions) take the streamed layout: per 128-entry slice m and K-chunk of 64 bytes per
    row, the precision's parts of [T1 | T2 | T3]^T, [m][chunk][part][128 x 64 B]. Decoded here,
    column kc*CK + j of slice m is the reference-tensor row of that K-column, to the split's
    accuracy, and zero in the padding."""
    got = image(coffee.BURGERS_JAC, k, cell, prec)
    if got is None:
        pytest.skip("no tensor-core kernel for this combination")
    img, meta = got
    mtiles, kbytes, kelems, K, parts, aexact, nca, _ = meta
    if kbytes != 64:
        pytest.skip("resident layout for this precision")
    tf32 = TF32[prec]
    d, ns = 2 + cell, coffee.nnodes(cell, k)
    nb, K1, P = ns * ns, ns * d, d * (d + 1) // 2
    ck = 16 if tf32 else 32
    KA1 = nca * ck
    ncd = kelems // ck
    assert aexact == 0 and parts == TPARTS[prec] and mtiles == math.ceil(nb / 128)
    assert KA1 == math.ceil(K1 / ck) * ck and kelems == math.ceil((KA1 + K1 + P) / ck) * ck
    tb = 128 * 64
    assert len(img) == mtiles * ncd * parts * tb
    T = coffee.reference_tensor(coffee.BURGERS_JAC, k, cell)
    u = 2.0 ** -11 if tf32 else 2.0 ** -8
    for m in range(mtiles):
        cols = []
        for kc in range(ncd):
            base = (m * ncd + kc) * parts * tb
            cols.append(sum(decode(img[base + q * tb:base + (q + 1) * tb], 64, tf32).astype(np.float64)
                            for q in range(parts)))
        A = np.hstack(cols)                                    # [128, ncd * ck]
        rows = slice(m * 128, min(nb, (m + 1) * 128))
        nr = rows.stop - rows.start
        assert not A[nr:].any()
        for kk in range(kelems):
            tr = (kk if kk < K1 else ns * d + kk - KA1 if KA1 <= kk < KA1 + K1
                  else 2 * ns * d + kk - KA1 - K1 if KA1 + K1 <= kk < KA1 + K1 + P else -1)
            if tr < 0:
                assert not A[:, kk].any(), kk
                continue
            want = T[tr, rows]
            assert np.all(np.abs(A[:nr, kk] - want) <= u ** parts * 1.01 * np.abs(want) + 1e-300), (m, kk)
