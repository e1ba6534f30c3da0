"""Host-only plans of the warm-start network's tensor-core convolutions (no GPU): the
invariants the kernels rely on -- every output voxel of a region written exactly once,
every staged read inside its stage, whole swizzle atoms, TMA box limits, TMEM and
shared-memory budgets, at most one wave of weight-gradient blocks -- for every layer of the
network and the shapes of the GPU parity tests, at several SM counts."""
import ctypes

import pytest

NETWORK = [((184, 128, 128), 16, 16, 27), ((184, 128, 128), 48, 16, 27), ((92, 64, 64), 16, 32, 27),
           ((92, 64, 64), 32, 32, 27), ((92, 64, 64), 96, 32, 27), ((46, 32, 32), 32, 64, 27),
           ((46, 32, 32), 64, 64, 27), ((46, 32, 32), 192, 64, 27), ((23, 16, 16), 64, 128, 27),
           ((23, 16, 16), 128, 128, 27), ((184, 128, 128), 16, 16, 1)]
CONV_SHAPES = [((4, 4, 8), 128, 16, 1), ((5, 7, 40), 16, 16, 27), ((4, 6, 24), 48, 48, 27), ((3, 5, 128), 16, 32, 27),
               ((3, 5, 200), 16, 32, 27), ((2, 3, 16), 16, 256, 27), ((5, 6, 32), 16, 16, 1),
               ((48, 128, 128), 16, 16, 27), ((24, 64, 64), 48, 128, 27), ((20, 32, 32), 64, 192, 27),
               ((3, 5, 256), 16, 32, 27), ((5, 7, 37), 16, 16, 27)]
WGRAD_SHAPES = [((3, 5, 32), 48, 16, 27), ((2, 3, 16), 16, 16, 27), ((1, 1, 16), 32, 48, 27),
                ((2, 2, 48), 192, 64, 27), ((2, 3, 16), 128, 256, 27), ((5, 4, 64), 16, 16, 27),
                ((4, 3, 32), 96, 32, 27), ((2, 2, 16), 1024, 16, 1), ((1, 2, 16), 512, 16, 27),
                ((24, 32, 64), 16, 16, 27)]


@pytest.fixture(scope="module")
def L():
    from paper_2211_03516_gb300 import build
    build.build()
    from paper_2211_03516_gb300 import vamrt
    lib = vamrt.lib()
    for f in (lib.vamrt_conv3d_halo_plan, lib.vamrt_conv3d_wgrad_plan):
        f.argtypes = [ctypes.c_int32] * 7 + [ctypes.c_void_p]
    return lib


def widest_block(c):
    return 64 if c % 64 == 0 else 32 if c % 32 == 0 else 16


@pytest.mark.parametrize("sms", [152, 148, 5])
@pytest.mark.parametrize("shape,cin,cout,taps", NETWORK + CONV_SHAPES)
def test_halo_plan_invariants(L, shape, cin, cout, taps, sms):
    D, H, W = shape
    out = (ctypes.c_int32 * 18)()
    assert L.vamrt_conv3d_halo_plan(D, H, W, cin, cout, taps, sms, ctypes.addressof(out)) == 0
    planned, TZ, TY, Nt, T, WP, PT, NX, rowtile, mg, adv, a_bytes, box_bytes, stage, ncols, ry, nslice, nitems = \
        list(out)
    if not planned:
        assert W % 8 or W + 16 > 256            # only the gather kernel's shapes
        return
    halo = 1 if taps == 27 else 0
    # one TMA box {16 channels, WP, TY + 2 halo, TZ + 2 halo} per chunk: dimensions <= 256
    assert WP == W + 16 and WP <= 256 and TY + 2 * halo <= 256 and TZ + 2 * halo <= 256
    assert WP % 8 == 0 and PT == (TY + 2 * halo) * WP
    assert box_bytes == (TZ + 2 * halo) * PT * 32 and a_bytes >= box_bytes and a_bytes % 256 == 0
    assert stage % 1024 == 0 and stage >= a_bytes + taps * Nt * 32 and 2 * stage <= 225 * 1024
    assert NX == (3 if taps == 27 else 1) and 2 * T * NX * Nt <= ncols <= 512 and ncols & (ncols - 1) == 0
    assert cout % Nt == 0 and nslice == cout // Nt and NX * Nt <= 256
    assert ry == -(-H // TY) and nitems == -(-D // TZ) * ry * nslice
    assert rowtile == (W == 128) and adv + 2 * mg <= 128
    # the kernel's tiles: starts, the rows each writes, and its (dz, dy)-shifted reads
    hits = {}
    for j in range(T):
        if rowtile:
            oz = j // TY
            q = oz * PT + (j - oz * TY) * WP + 8
        else:
            per = -(-(TY * WP) // adv)
            oz = j // per
            q = oz * PT + adv * (j - oz * per)
        assert q % 8 == 0                            # whole 256-byte swizzle atoms
        for dz in ((-1, 0, 1) if halo else (0,)):
            for dy in ((-1, 0, 1) if halo else (0,)):
                lo = halo * (PT + WP) + q + dz * PT + dy * WP
                assert lo >= 0 and (lo + 128) * 32 <= a_bytes
        for t in range(128):
            qq = q + t
            ozz = qq // PT
            rem = qq - ozz * PT
            oy = rem // WP
            x = rem - oy * WP - 8
            if mg <= t < mg + adv and ozz == oz and oy < TY and 0 <= x < W:
                hits[(ozz, oy, x)] = hits.get((ozz, oy, x), 0) + 1
                if taps == 27 and not rowtile:
                    assert 1 <= t <= 126              # both dx neighbours inside the tile
    assert hits == {(z, y, x): 1 for z in range(TZ) for y in range(TY) for x in range(W)}


@pytest.mark.parametrize("sms", [152, 148, 3])
@pytest.mark.parametrize("shape,cin,cout,taps", NETWORK + WGRAD_SHAPES)
def test_wgrad_plan_invariants(L, shape, cin, cout, taps, sms):
    D, H, W = shape
    if W % 16:
        pytest.skip("the weight gradient takes W % 16 == 0")
    out = (ctypes.c_int32 * 17)()
    assert L.vamrt_conv3d_wgrad_plan(D, H, W, cin, cout, taps, sms, ctypes.addressof(out)) == 0
    planned, Mtot, nmt, tpg, kp, KS, BX, nstage, cwA, cwB, slots, slot_bytes, per_sm, ncols, ngroups, nsplit, spb = \
        list(out)
    assert planned == 1
    P = D * H * W
    assert Mtot == taps * cin and nmt == -(-Mtot // 128)
    assert KS == (64 if W % 64 == 0 else 32) and BX >= 16 and W % BX == 0 and KS % BX == 0
    assert nstage == -(-P // KS)
    assert cwA == widest_block(cin) and cwB == widest_block(cout)
    # a slot: the dY column blocks, then 128 tpg rows of X^T, KS positions each
    assert slot_bytes % 1024 == 0 and slot_bytes >= (cout + 128 * tpg) * KS * 2
    budget = 108 * 1024 if per_sm == 2 else 220 * 1024
    assert per_sm in (1, 2) and 3 <= slots <= 4 and slots * slot_bytes <= budget
    assert 1 <= kp <= KS // 16 and tpg * kp * cout <= ncols <= 512 // per_sm and ncols & (ncols - 1) == 0
    # tile groups cover the M tiles, blocks the positions, at most one wave
    assert 1 <= tpg <= 8 and ngroups == -(-nmt // tpg) and (ngroups - 1) * tpg < nmt
    assert nsplit * spb >= nstage and (nsplit - 1) * spb < nstage
    assert ngroups * nsplit <= max(per_sm * sms, ngroups)
    # TMA destinations and MMA start addresses on whole swizzle atoms
    atom = {16: 256, 32: 512, 64: 1024}
    assert (KS * 2 * cwA) % 1024 == 0 and (KS * 2 * cwB) % 1024 == 0
    assert (BX * 2 * cwA) % atom[cwA] == 0 and (16 * 2 * cwA) % atom[cwA] == 0 and (16 * 2 * cwB) % atom[cwB] == 0


def test_plans_reject_bad_arguments(L):
    from paper_2211_03516_gb300 import vamrt
    out = (ctypes.c_int32 * 18)()
    assert L.vamrt_conv3d_halo_plan(4, 4, 16, 16, 16, 27, 0, ctypes.addressof(out)) == vamrt.VAMRT_EINVAL
    assert L.vamrt_conv3d_wgrad_plan(4, 4, 16, 16, 16, 27, 152, None) == vamrt.VAMRT_EINVAL
    assert L.vamrt_conv3d_wgrad_plan(4, 4, 24, 16, 16, 27, 152, ctypes.addressof(out)) == 0 and out[0] == 0
