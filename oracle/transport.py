"""Oracle: cell transmissions and transport solves (test infrastructure only).

* `transmit` -- the FP64 random-walk cell transmission of the Monte Carlo
  method section (Eq. 4-6), canonical frame: entry on the left face at
  y = xi tau with direction (cos, sin); analog (survival c) or implicit
  capture. Implemented in C (walk.c).
* `solve_analog` -- standard Monte Carlo with implicit capture on a grid,
  one history at a time, track-length flux tally (Eq. 5-7). C (solve.c).
* `solve_gmc` -- the four-stage GMC transport algorithm, one wave of live
  particles at a time:
    1. rotate each particle's state into the canonical left-entry frame;
    2. draw z ~ N(0, I) and sample the exit state (or, for pinning the loop,
       run the random walk in that frame instead);
    3. attenuate by exp(-sigma_a s) and tally Delta w / (V sigma_a);
    4. rotate the exit back to global coordinates and cross into the
       neighbour; stop at the domain edge, roulette below the weight cutoff.
  Births in a source cell are walked to their first face crossing with the
  random walk, or, given an internal sampler (the paper's internal model for
  volumetric sources), their exit from the birth cell is sampled by it.
  Variants: a surface source on the left boundary (`wall=`), x-y geometry
  with 3-D directions carried as their projection on the plane
  (`geometry="xy"`), and cells cut into rectangles dx x dy (`solve_gmc_rect`);
  cells outside a network's training box are sampled at their
  scattering-equivalent condition (`equivalent_condition`,
  `equivalent_condition_rect`) or walked.

Global faces use the same counter-clockwise numbering as a cell in its own
frame: 0 = south (y-), 1 = east (x+), 2 = north (y+), 3 = west (x-). A
particle entering through global face F is seen in the frame rotated by
r = (F + 1) mod 4 quarter turns, which maps the canonical left face (3) onto
F; canonical face f maps to global face (f + r) mod 4 with the same
counter-clockwise parameter q, and directions rotate by r quarter turns.
Crossing face G at parameter q enters the neighbour through face (G + 2) mod 4
with canonical entry position xi = q.
"""
import ctypes

import numpy as np

from ._clib import lib
from . import rng
from . import mlp

MODE_ANALOG = 0
MODE_IMPLICIT = 1


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def transmit(xi, cos_in, sin_in, tau, c, mode, seed, ids=None, events=None, id0=0, ctr0=0):
    """Batched canonical-frame random-walk transmission in FP64."""
    xi, cos_in, sin_in, tau, c = (_c(a, np.float64) for a in (xi, cos_in, sin_in, tau, c))
    n = xi.shape[0]
    out = {k: np.zeros(n, dtype=np.float64) for k in ("q", "ux", "uy", "s")}
    status = np.zeros(n, dtype=np.int32)
    face = np.zeros(n, dtype=np.int32)
    ncoll = np.zeros(n, dtype=np.int64)
    if ids is None:
        lib().orc_transmit_batch(n, xi.ctypes.data, cos_in.ctypes.data, sin_in.ctypes.data,
                                 tau.ctypes.data, c.ctypes.data, mode, seed, id0, ctr0,
                                 status.ctypes.data, face.ctypes.data, out["q"].ctypes.data,
                                 out["ux"].ctypes.data, out["uy"].ctypes.data,
                                 out["s"].ctypes.data, ncoll.ctypes.data)
        ev = None
    else:
        ids = _c(ids, np.uint64)
        events = _c(events, np.uint32)
        ev = np.zeros(n, dtype=np.uint32)
        lib().orc_transmit_ids(n, xi.ctypes.data, cos_in.ctypes.data, sin_in.ctypes.data,
                               tau.ctypes.data, c.ctypes.data, mode, seed, ids.ctypes.data,
                               events.ctypes.data, status.ctypes.data, face.ctypes.data,
                               out["q"].ctypes.data, out["ux"].ctypes.data,
                               out["uy"].ctypes.data, out["s"].ctypes.data, ncoll.ctypes.data,
                               ev.ctypes.data)
    out.update(status=status, face=face, ncoll=ncoll, events=ev)
    return out


def transmit_rect(xi, cos_in, sin_in, tx, ty, c, mode, seed, ids=None, events=None):
    """transmit for rectangular cells (geometry variant): optical width tx,
    height ty, entry on the left face at y = xi ty; q normalized per face.
    Per-particle Philox ids (default 0..n-1) and first events (default 0)."""
    xi, cos_in, sin_in, tx, ty, c = (_c(a, np.float64) for a in (xi, cos_in, sin_in, tx, ty, c))
    n = xi.shape[0]
    ids = _c(np.arange(n) if ids is None else ids, np.uint64)
    events = _c(np.zeros(n) if events is None else events, np.uint32)
    out = {k: np.zeros(n, dtype=np.float64) for k in ("q", "ux", "uy", "s")}
    status = np.zeros(n, dtype=np.int32)
    face = np.zeros(n, dtype=np.int32)
    ncoll = np.zeros(n, dtype=np.int64)
    ev = np.zeros(n, dtype=np.uint32)
    lib().orc_transmit_rect_ids(n, xi.ctypes.data, cos_in.ctypes.data, sin_in.ctypes.data,
                                tx.ctypes.data, ty.ctypes.data, c.ctypes.data, mode, seed,
                                ids.ctypes.data, events.ctypes.data, status.ctypes.data,
                                face.ctypes.data, out["q"].ctypes.data, out["ux"].ctypes.data,
                                out["uy"].ctypes.data, out["s"].ctypes.data, ncoll.ctypes.data,
                                ev.ctypes.data)
    out.update(status=status, face=face, ncoll=ncoll, events=ev)
    return out


def transmit_xy(xi, ux_in, uy_in, uz_in, tx, ty, c, mode, seed, ids=None, events=None,
                sphere=True):
    """Transmission in x-y geometry (geometry variant: the cell is the
    cross-section of an infinite prism, directions are 3-D unit vectors, s is
    the 3-D track length): entry on the left face at y = xi ty with direction
    (ux_in, uy_in, uz_in); scattering isotropic on the sphere (on the circle
    with sphere=False, which is transmit_rect draw for draw). The exit
    direction's projection (ux, uy) lies in the unit disk."""
    xi, ux_in, uy_in, uz_in, tx, ty, c = (_c(a, np.float64)
                                          for a in (xi, ux_in, uy_in, uz_in, tx, ty, c))
    n = xi.shape[0]
    ids = _c(np.arange(n) if ids is None else ids, np.uint64)
    events = _c(np.zeros(n) if events is None else events, np.uint32)
    out = {k: np.zeros(n, dtype=np.float64) for k in ("q", "ux", "uy", "uz", "s")}
    status = np.zeros(n, dtype=np.int32)
    face = np.zeros(n, dtype=np.int32)
    ncoll = np.zeros(n, dtype=np.int64)
    ev = np.zeros(n, dtype=np.uint32)
    lib().orc_transmit_xy_ids(n, xi.ctypes.data, ux_in.ctypes.data, uy_in.ctypes.data,
                              uz_in.ctypes.data, tx.ctypes.data, ty.ctypes.data, c.ctypes.data,
                              mode, int(bool(sphere)), seed, ids.ctypes.data, events.ctypes.data,
                              status.ctypes.data, face.ctypes.data, out["q"].ctypes.data,
                              out["ux"].ctypes.data, out["uy"].ctypes.data, out["uz"].ctypes.data,
                              out["s"].ctypes.data, ncoll.ctypes.data, ev.ctypes.data)
    out.update(status=status, face=face, ncoll=ncoll, events=ev)
    return out


def training_pairs_rect(xi, cos_in, sin_in, tau_x, tau_y, c, seed, ids=None):
    """Training pairs of a boundary model for rectangular cells (geometry
    variant with unequal sides): condition (xi, cos, sin, ln tau_x, c,
    ln(tau_y / tau_x)) [6, n], the aspect ratio as the sixth input, and
    target (p, cos_out, sin_out, ln s) [4, n] of the implicit-capture walk in
    the rectangle, p = face + q with q normalized per face."""
    xi, cos_in, sin_in, tau_x, tau_y, c = (np.asarray(a, dtype=np.float64)
                                           for a in (xi, cos_in, sin_in, tau_x, tau_y, c))
    r = transmit_rect(xi, cos_in, sin_in, tau_x, tau_y, c, MODE_IMPLICIT, seed, ids=ids)
    cond = np.stack([xi, cos_in, sin_in, np.log(tau_x), c, np.log(tau_y / tau_x)])
    y = np.stack([r["face"] + r["q"], r["ux"], r["uy"], np.log(r["s"])])
    return cond, y


def training_pairs_xy(xi, ux_in, uy_in, tau, c, seed, ids=None):
    """Training pairs of the boundary model in x-y geometry ("Network
    Architecture and Inputs": pure-scattering walks from the entry face, the
    direction encoded by its projection on the unit disk): condition
    (xi, ux_in, uy_in, ln tau, c) [5, n] and target (p, ux, uy, ln s) [4, n]
    of the implicit-capture 3-D walk, p = face + q. The out-of-plane entry
    component is sqrt(1 - ux_in^2 - uy_in^2) (its sign does not enter)."""
    xi, ux_in, uy_in, tau, c = (np.asarray(a, dtype=np.float64)
                                for a in (xi, ux_in, uy_in, tau, c))
    uz_in = np.sqrt(np.maximum(1.0 - ux_in * ux_in - uy_in * uy_in, 0.0))
    r = transmit_xy(xi, ux_in, uy_in, uz_in, tau, tau, c, MODE_IMPLICIT, seed, ids=ids)
    cond = np.stack([xi, ux_in, uy_in, np.log(tau), c])
    y = np.stack([r["face"] + r["q"], r["ux"], r["uy"], np.log(r["s"])])
    return cond, y


def walk_one(tau, c, mode, x, y, ux, uy, seed, pid, event0):
    """One random walk from an arbitrary point (cell frame, optical units)."""
    status = ctypes.c_int32()
    face = ctypes.c_int32()
    ncoll = ctypes.c_int64()
    ev = ctypes.c_uint32()
    out = np.zeros(6, dtype=np.float64)
    lib().orc_walk_one(float(tau), float(c), mode, float(x), float(y), float(ux), float(uy),
                       seed, int(pid), int(event0), ctypes.byref(status), ctypes.byref(face),
                       out.ctypes.data, ctypes.byref(ncoll), ctypes.byref(ev))
    return {"status": status.value, "face": face.value, "q": out[0], "x": out[1], "y": out[2],
            "ux": out[3], "uy": out[4], "s": out[5], "ncoll": ncoll.value, "event": ev.value}


def walk_one_xy(tau, c, mode, x, y, ux, uy, seed, pid, event0):
    """One random walk in x-y geometry (the cell is the cross-section of an
    infinite prism, directions are 3-D and scatter isotropically on the
    sphere) from an arbitrary point; (ux, uy) is the direction's projection
    on the plane, s the 3-D track length. Same outputs as walk_one."""
    status = ctypes.c_int32()
    face = ctypes.c_int32()
    ncoll = ctypes.c_int64()
    ev = ctypes.c_uint32()
    out = np.zeros(6, dtype=np.float64)
    lib().orc_walk_one_xy(float(tau), float(c), mode, float(x), float(y), float(ux), float(uy),
                          seed, int(pid), int(event0), ctypes.byref(status), ctypes.byref(face),
                          out.ctypes.data, ctypes.byref(ncoll), ctypes.byref(ev))
    return {"status": status.value, "face": face.value, "q": out[0], "x": out[1], "y": out[2],
            "ux": out[3], "uy": out[4], "s": out[5], "ncoll": ncoll.value, "event": ev.value}


def solve_analog(tau, c, src, n_hist, seed, w_cut=1e-4, p_survive=0.1):
    """Standard MC solve; tau, c, src are [ny, nx]. Returns (flux [ny, nx], stats dict)."""
    tau, c, src = (_c(a, np.float64) for a in (tau, c, src))
    ny, nx = tau.shape
    flux = np.zeros((ny, nx), dtype=np.float64)
    st = np.zeros(6, dtype=np.float64)
    rc = lib().orc_solve_analog(nx, ny, tau.ctypes.data, c.ctypes.data, src.ctypes.data,
                                n_hist, seed, w_cut, p_survive, flux.ctypes.data, st.ctypes.data)
    if rc != 0:
        raise ValueError("orc_solve_analog failed: %d" % rc)
    return flux, _stats(st)


def _stats(st):
    return {"leak": st[0], "absorbed": st[1], "roulette_net": st[2], "transmissions": st[3],
            "collisions": st[4], "roulette_kills": st[5]}


def rot(ux, uy, k):
    """Rotate direction(s) by k quarter turns counter-clockwise."""
    k = np.mod(k, 4)
    rx = np.select([k == 0, k == 1, k == 2, k == 3], [ux, -uy, -ux, uy])
    ry = np.select([k == 0, k == 1, k == 2, k == 3], [uy, ux, -uy, -ux])
    return rx, ry


def deposit(w, s, tau, c):
    """Delta w of Eq. 6 and the Eq. 7 flux score for track length s (optical units)."""
    a = 1.0 - c
    pos = a > 0.0
    a_safe = np.where(pos, a, 1.0)
    dw = np.where(pos, w * (-np.expm1(-a_safe * s)), 0.0)
    score = np.where(pos, dw / (a_safe * tau), w * s / tau)
    return dw, score


def mlp_sampler(net, steps, integrator, seed):
    """Stage 2 with the flow ODE: noise at (id, event, TAG_NOISE), one event used."""
    def f(xi, cos_c, sin_c, tau, c, ids, events, rot=None):
        cond = np.stack([xi, cos_c, sin_c, np.log(tau), c])
        z = rng.normals_for(seed, ids, events, rng.TAG_NOISE)
        d = mlp.decode(net, mlp.sample(net, cond, z, steps, integrator))
        return d["face"], d["q"], d["ux"], d["uy"], d["s"], np.asarray(events, np.uint32) + 1
    return f


def mlp_sampler_xy(net, steps, integrator, seed):
    """Stage 2 in x-y geometry with the x-y boundary network: the condition
    holds the projected entry direction, exits are decoded into the unit
    disk (decode_disk)."""
    def f(xi, ux_c, uy_c, tau, c, ids, events, rot=None):
        cond = np.stack([xi, ux_c, uy_c, np.log(tau), c])
        z = rng.normals_for(seed, ids, events, rng.TAG_NOISE)
        d = mlp.decode_disk(net, mlp.sample(net, cond, z, steps, integrator))
        return d["face"], d["q"], d["ux"], d["uy"], d["s"], np.asarray(events, np.uint32) + 1
    return f


def walk_sampler_xy(seed):
    """Stage 2 in x-y geometry replaced by the walk the x-y training pairs
    take (transmit_xy in the canonical frame, out-of-plane entry component
    sqrt(1 - ux^2 - uy^2) from the handed-over projection)."""
    def f(xi, ux_c, uy_c, tau, c, ids, events, rot=None):
        ux_c, uy_c = np.asarray(ux_c, np.float64), np.asarray(uy_c, np.float64)
        uz = np.sqrt(np.maximum(1.0 - ux_c * ux_c - uy_c * uy_c, 0.0))
        r = transmit_xy(xi, ux_c, uy_c, uz, tau, tau, c, MODE_IMPLICIT, seed, ids=ids,
                        events=events)
        return r["face"], r["q"], r["ux"], r["uy"], r["s"], r["events"]
    return f


def walk_sampler(seed):
    """Stage 2 replaced by the implicit-capture random walk in the canonical frame."""
    def f(xi, cos_c, sin_c, tau, c, ids, events, rot=None):
        r = transmit(xi, cos_c, sin_c, tau, c, MODE_IMPLICIT, seed, ids=ids, events=events)
        return r["face"], r["q"], r["ux"], r["uy"], r["s"], r["events"]
    return f


def equivalent_condition(tau, c, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """Scattering-equivalent condition of cells (tau, c) inside a network's
    training box [tau_lo, tau_hi] x [c_lo, c_hi].

    The implicit-capture walk (MC section, Eq. 4; absorption applied
    afterwards as exp(-(1 - c) s), Eq. 5) draws flights at rate c in a cell of
    side tau, which is the walk at rate 1 in a cell of side c tau with every
    length divided by c: exits depend on the scattering thickness c tau only,
    and track lengths scale as 1 / c. A cell (tau', c') with c' tau' = c tau
    therefore has the same exit law, and s = s' c' / c. c' is c moved into
    [c_lo, c_hi] and [c tau / tau_hi, c tau / tau_lo]; cells inside the box
    keep (tau, c). Returns (tau', c', ok); ok is False where no equivalent
    exists (c tau outside [c_lo tau_lo, c_hi tau_hi], c = 0 included), and
    those cells keep (tau, c)."""
    tau = np.asarray(tau, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    (t_lo, t_hi), (c_lo, c_hi) = tau_range, c_range
    w = c * tau
    lo = np.maximum(c_lo, w / t_hi)
    hi = np.minimum(c_hi, w / t_lo)
    ok = (w > 0.0) & (lo <= hi)
    inside = (tau >= t_lo) & (tau <= t_hi) & (c >= c_lo) & (c <= c_hi)
    ok = ok | inside
    cp = np.where(inside, c, np.where(ok, np.clip(c, lo, np.maximum(lo, hi)), c))
    tp = np.where(inside | ~ok, tau, np.clip(w / np.where(ok, cp, 1.0), t_lo, t_hi))
    return tp, cp, ok


def equivalent_sampler(sampler, fallback, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """Stage 2 for grids whose cells leave the network's training box: each
    particle is sampled by `sampler` at its cell's scattering-equivalent
    condition (equivalent_condition) and its track length scaled by c' / c;
    particles in cells without an equivalent go to `fallback` (the random
    walk) at their own (tau, c). Inside the box this is `sampler` itself."""
    def f(xi, cos_c, sin_c, tau, c, ids, events, rot=None):
        xi, cos_c, sin_c, tau, c = (np.asarray(a, dtype=np.float64)
                                    for a in (xi, cos_c, sin_c, tau, c))
        ids = np.asarray(ids, dtype=np.uint64)
        events = np.asarray(events, dtype=np.uint32)
        tp, cp, ok = equivalent_condition(tau, c, tau_range, c_range)
        n = xi.shape[0]
        face = np.zeros(n, np.int64)
        q, ux, uy, s = (np.zeros(n) for _ in range(4))
        ev = np.zeros(n, np.uint32)
        for sel, fn, tt, cc in ((ok, sampler, tp, cp), (~ok, fallback, tau, c)):
            k = np.nonzero(sel)[0]
            if k.size == 0:
                continue
            r = None if rot is None else np.asarray(rot)[k]
            fa, qa, uxa, uya, sa, eva = fn(xi[k], cos_c[k], sin_c[k], tt[k], cc[k], ids[k],
                                           events[k], rot=r)
            face[k], q[k], ux[k], uy[k], ev[k] = fa, qa, uxa, uya, eva
            s[k] = np.asarray(sa) * (cc[k] / c[k]) if fn is sampler else sa
        return face, q, ux, uy, s, ev
    return f


def equivalent_internal_sampler(internal, fallback, tau_range=(0.1, 1000.0),
                                c_range=(0.5, 0.999)):
    """Births for grids whose cells leave the internal model's training box:
    the same reading as equivalent_sampler. A birth at the normalized point
    (X, Y) of a cell (tau, c) walks, in cell units, exactly as a birth at
    (X, Y) of a cell (tau', c') with c' tau' = c tau (flights at rate c in
    side tau are flights at rate c' in side tau', every length times c'/c),
    so births in cells with an equivalent are sampled by `internal` at
    (tau', c') with s scaled by c'/c; births in cells without one go to
    `fallback` (the walk) at their own (tau, c)."""
    def f(X, Y, tau, c, ids, u_angle):
        X, Y, tau, c = (np.asarray(a, dtype=np.float64) for a in (X, Y, tau, c))
        ids = np.asarray(ids, dtype=np.uint64)
        u_angle = np.asarray(u_angle, dtype=np.float64)
        tp, cp, ok = equivalent_condition(tau, c, tau_range, c_range)
        n = X.shape[0]
        face = np.zeros(n, np.int64)
        q, ux, uy, s = (np.zeros(n) for _ in range(4))
        ev = np.zeros(n, np.uint32)
        for sel, fn, tt, cc in ((ok, internal, tp, cp), (~ok, fallback, tau, c)):
            k = np.nonzero(sel)[0]
            if k.size == 0:
                continue
            fa, qa, uxa, uya, sa, eva = fn(X[k], Y[k], tt[k], cc[k], ids[k], u_angle[k])
            face[k], q[k], ux[k], uy[k], ev[k] = fa, qa, uxa, uya, eva
            s[k] = np.asarray(sa) * (cc[k] / c[k]) if fn is internal else sa
        return face, q, ux, uy, s, ev
    return f


def internal_condition(X, Y, tau, c):
    """Condition of the internal model for births at (X, Y) in [0,1]^2 of a cell:
    (X, Y, ln tau, c, distance to the nearest face in cell units) -> [5, B]."""
    X, Y, tau, c = (np.asarray(a, dtype=np.float64) for a in (X, Y, tau, c))
    d = np.minimum(np.minimum(X, Y), np.minimum(1.0 - X, 1.0 - Y))
    return np.stack([X, Y, np.log(tau), c, d])


def mlp_internal_sampler(net, steps, integrator, seed):
    """Births with the internal model: exit (cell frame) from the flow ODE with
    noise at (id, 0, TAG_NOISE); the next event is 1."""
    def f(X, Y, tau, c, ids, u_angle):
        cond = internal_condition(X, Y, tau, c)
        ids = np.asarray(ids, np.uint64)
        z = rng.normals_for(seed, ids, np.zeros(ids.size, np.uint32), rng.TAG_NOISE)
        d = mlp.decode(net, mlp.sample(net, cond, z, steps, integrator))
        return d["face"], d["q"], d["ux"], d["uy"], d["s"], np.ones(ids.size, np.uint32)
    return f


def walk_internal_sampler(seed):
    """Births walked exactly as the random-walk solve does: direction from the
    birth draw, implicit-capture walk from event 0."""
    def f(X, Y, tau, c, ids, u_angle):
        out = [np.zeros(len(ids)) for _ in range(5)] + [np.zeros(len(ids), np.uint32)]
        for k in range(len(ids)):
            ang = 2.0 * np.pi * u_angle[k]
            r = walk_one(tau[k], c[k], MODE_IMPLICIT, X[k] * tau[k], Y[k] * tau[k], np.cos(ang),
                         np.sin(ang), seed, int(ids[k]), 0)
            for a, v in zip(out, (r["face"], r["q"], r["ux"], r["uy"], r["s"], r["event"])):
                a[k] = v
        return out[0].astype(np.int64), out[1], out[2], out[3], out[4], out[5]
    return f


def internal_pairs(n, seed, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """Training pairs of the internal model ("Network Architecture and
    Inputs": births inside a cell, the implicit-capture walk to the exit):
    for sample i, the draw (i, 0, tag 7) gives ln tau uniform in the log
    range, c uniform, X and Y uniform; (i, 1, tag 7) the birth direction at
    angle 2 pi u0 on the circle; the walk draws from event 2. Returns cond
    [5, n] (internal_condition) and y [4, n] = (p, ux, uy, ln s) in the
    cell's own frame, in FP64."""
    ids = np.arange(n, dtype=np.uint64)
    u0 = rng.uniforms_for(seed, ids, np.zeros(n, np.uint32), 7)
    u1 = rng.uniforms_for(seed, ids, np.ones(n, np.uint32), 7)
    lo, hi = np.log(tau_range[0]), np.log(tau_range[1])
    tau = np.exp(lo + (hi - lo) * u0[0])
    c = c_range[0] + (c_range[1] - c_range[0]) * u0[1]
    X, Y = u0[2], u0[3]
    ang = 2.0 * np.pi * u1[0]
    y = np.zeros((4, n))
    for i in range(n):
        w = walk_one(tau[i], c[i], MODE_IMPLICIT, X[i] * tau[i], Y[i] * tau[i], np.cos(ang[i]),
                     np.sin(ang[i]), seed, i, 2)
        y[:, i] = (w["face"] + w["q"], w["ux"], w["uy"], np.log(max(w["s"], mlp.S_MIN)))
    return internal_condition(X, Y, tau, c), y


def mlp_internal_sampler_xy(net, steps, integrator, seed):
    """mlp_internal_sampler for x-y geometry: the x-y internal model's exit,
    decoded into the unit disk (decode_disk)."""
    def f(X, Y, tau, c, ids, u_angle):
        cond = internal_condition(X, Y, tau, c)
        ids = np.asarray(ids, np.uint64)
        z = rng.normals_for(seed, ids, np.zeros(ids.size, np.uint32), rng.TAG_NOISE)
        d = mlp.decode_disk(net, mlp.sample(net, cond, z, steps, integrator))
        return d["face"], d["q"], d["ux"], d["uy"], d["s"], np.ones(ids.size, np.uint32)
    return f


def walk_internal_sampler_xy(seed):
    """Births of an x-y solve walked as the random-walk solve walks them:
    direction on the sphere (birth_directions), walk_one_xy from event 0."""
    def f(X, Y, tau, c, ids, u_angle):
        ids = np.asarray(ids, np.uint64)
        bux, buy = birth_directions(seed, ids, u_angle, "xy")
        out = [np.zeros(len(ids)) for _ in range(5)] + [np.zeros(len(ids), np.uint32)]
        for k in range(len(ids)):
            r = walk_one_xy(tau[k], c[k], MODE_IMPLICIT, X[k] * tau[k], Y[k] * tau[k], bux[k],
                            buy[k], seed, int(ids[k]), 0)
            for a, v in zip(out, (r["face"], r["q"], r["ux"], r["uy"], r["s"], r["event"])):
                a[k] = v
        return out[0].astype(np.int64), out[1], out[2], out[3], out[4], out[5]
    return f


def internal_pairs_xy(n, seed, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """Training pairs of the x-y internal model (births inside a prism cell,
    3-D isotropic direction, implicit-capture walk to the exit): for sample
    i, the draw (i, 0, tag 9) gives ln tau uniform in the log range, c
    uniform, X and Y uniform; (i, 1, tag 9) the direction, azimuth 2 pi u0 and
    polar cosine 2 u1 - 1, projected on the plane; the walk draws from event
    2. Returns cond [5, n] = (X, Y, ln tau, c, distance to the nearest face)
    and y [4, n] = (p, ux, uy, ln s) in the cell's own frame, in FP64."""
    ids = np.arange(n, dtype=np.uint64)
    u0 = rng.uniforms_for(seed, ids, np.zeros(n, np.uint32), 9)
    u1 = rng.uniforms_for(seed, ids, np.ones(n, np.uint32), 9)
    lo, hi = np.log(tau_range[0]), np.log(tau_range[1])
    ltau = lo + (hi - lo) * u0[0]
    c = c_range[0] + (c_range[1] - c_range[0]) * u0[1]
    X, Y = u0[2], u0[3]
    mu = 2.0 * u1[1] - 1.0
    r = np.sqrt(np.maximum(1.0 - mu * mu, 0.0))
    ux, uy = r * np.cos(2.0 * np.pi * u1[0]), r * np.sin(2.0 * np.pi * u1[0])
    tau = np.exp(ltau)
    y = np.zeros((4, n))
    for i in range(n):
        w = walk_one_xy(tau[i], c[i], MODE_IMPLICIT, X[i] * tau[i], Y[i] * tau[i], ux[i], uy[i],
                        seed, i, 2)
        y[:, i] = (w["face"] + w["q"], w["ux"], w["uy"], np.log(max(w["s"], mlp.S_MIN)))
    cond = internal_condition(X, Y, tau, c)
    return cond, y


def walk_sampler_global(seed):
    """Stage 2 replaced by the implicit-capture walk in the cell's own (global)
    frame, as a random-walk solve takes it: entry face F = (rot - 1) mod 4 at
    counter-clockwise parameter 1 - xi, global direction rot(canonical, rot);
    the exit is returned in the canonical frame (face - rot, same q, direction
    rotated back)."""
    def f(xi, cos_c, sin_c, tau, c, ids, events, rot=None):
        n = len(ids)
        face = np.zeros(n, np.int64)
        out = [np.zeros(n) for _ in range(4)]
        ev = np.zeros(n, np.uint32)
        for k in range(n):
            r = int(rot[k])
            F = (r - 1) % 4
            x = float(xi[k])
            X, Y = {0: (1.0 - x, 0.0), 1: (1.0, 1.0 - x), 2: (x, 1.0), 3: (0.0, x)}[F]
            gx, gy = rot_dir(cos_c[k], sin_c[k], r)
            w = walk_one(tau[k], c[k], MODE_IMPLICIT, X * tau[k], Y * tau[k], gx, gy, seed,
                         int(ids[k]), int(events[k]))
            face[k] = (w["face"] - r) % 4
            ux, uy = rot_dir(w["ux"], w["uy"], -r)
            out[0][k], out[1][k], out[2][k], out[3][k] = w["q"], ux, uy, w["s"]
            ev[k] = w["event"]
        return face, out[0], out[1], out[2], out[3], ev
    return f


def walk_sampler_global_xy(seed):
    """walk_sampler_global in x-y geometry (walk_one_xy): the random walk a
    random-walk x-y solve takes through a cell, in the cell's own frame."""
    def f(xi, ux_c, uy_c, tau, c, ids, events, rot=None):
        n = len(ids)
        face = np.zeros(n, np.int64)
        out = [np.zeros(n) for _ in range(4)]
        ev = np.zeros(n, np.uint32)
        for k in range(n):
            r = int(rot[k])
            F = (r - 1) % 4
            x = float(xi[k])
            X, Y = {0: (1.0 - x, 0.0), 1: (1.0, 1.0 - x), 2: (x, 1.0), 3: (0.0, x)}[F]
            gx, gy = rot_dir(ux_c[k], uy_c[k], r)
            w = walk_one_xy(tau[k], c[k], MODE_IMPLICIT, X * tau[k], Y * tau[k], gx, gy, seed,
                            int(ids[k]), int(events[k]))
            face[k] = (w["face"] - r) % 4
            ux, uy = rot_dir(w["ux"], w["uy"], -r)
            out[0][k], out[1][k], out[2][k], out[3][k] = w["q"], ux, uy, w["s"]
            ev[k] = w["event"]
        return face, out[0], out[1], out[2], out[3], ev
    return f


def rot_dir(ux, uy, k):
    """Scalar form of rot."""
    rx, ry = rot(np.array([ux]), np.array([uy]), k)
    return float(rx[0]), float(ry[0])


def wall_births(wall, n_hist, seed):
    """Histories of an isotropic surface source on the left boundary (x = 0),
    from the birth draw (id, 0, TAG_BIRTH) = (u0, u1, u2, u3): boundary cell
    row j with probability wall[j] / sum(wall) (first row whose cumulative
    strength reaches u0 * total), entry point y = j + u1 on the cell's left
    face, and the cosine law for the direction (the flux of an isotropic
    radiance through a surface): sin(theta) = 2 u2 - 1, cos(theta) =
    sqrt(1 - sin^2) > 0. Returns (j, xi, gx, gy) per history."""
    cdf = np.cumsum(np.maximum(np.asarray(wall, dtype=np.float64), 0.0))
    ids = np.arange(n_hist, dtype=np.uint64)
    ub = rng.uniforms_for(seed, ids, np.zeros(n_hist, np.uint32), rng.TAG_BIRTH)
    j = np.searchsorted(cdf, ub[0] * cdf[-1], side="left")
    sn = 2.0 * ub[2] - 1.0
    return j, ub[1], np.sqrt(np.maximum(1.0 - sn * sn, 0.0)), sn


def wall_births_xy(wall, n_hist, seed):
    """wall_births in x-y geometry: row j and entry point from u0, u1 as
    there; the 3-D cosine law for the direction, cosine to the inward normal
    mu = sqrt(u2) and azimuth about it 2 pi u3, so the projected entry
    direction is (mu, sqrt(1 - mu^2) cos(2 pi u3))."""
    cdf = np.cumsum(np.maximum(np.asarray(wall, dtype=np.float64), 0.0))
    ids = np.arange(n_hist, dtype=np.uint64)
    ub = rng.uniforms_for(seed, ids, np.zeros(n_hist, np.uint32), rng.TAG_BIRTH)
    j = np.searchsorted(cdf, ub[0] * cdf[-1], side="left")
    mu = np.sqrt(ub[2])
    return j, ub[1], mu, np.sqrt(np.maximum(1.0 - mu * mu, 0.0)) * np.cos(2.0 * np.pi * ub[3])


def birth_directions(seed, ids, u_angle, geometry):
    """Direction of a volumetric birth (isotropic): on the circle at angle
    2 pi u_angle (flat), or on the sphere (xy) with that azimuth and polar
    cosine 2 u - 1, u the first uniform of the draw (id, 1, TAG_BIRTH),
    projected on the plane."""
    ang = 2.0 * np.pi * np.asarray(u_angle, np.float64)
    if geometry == "flat":
        return np.cos(ang), np.sin(ang)
    ids = np.asarray(ids, np.uint64)
    u = rng.uniforms_for(seed, ids, np.ones(ids.size, np.uint32), rng.TAG_BIRTH)[0]
    mu = 2.0 * u - 1.0
    r = np.sqrt(np.maximum(1.0 - mu * mu, 0.0))
    return r * np.cos(ang), r * np.sin(ang)


def solve_gmc(tau, c, src, n_hist, seed, sampler, w_cut=1e-4, p_survive=0.1, max_waves=100000,
              internal=None, wall=None, geometry="flat"):
    """Event-based GMC solve; tau, c, src are [ny, nx]. Returns (flux, stats).

    internal: sampler of births (mlp_internal_sampler / walk_internal_sampler),
    or None to walk every birth with walk_one.
    wall: [ny] strengths of a surface source on the left boundary instead of
    the volumetric source src (see wall_births); each history enters its
    boundary cell through the west face with weight 1 and next event 0.
    geometry: "flat" (directions on the circle) or "xy" (x-y geometry: every
    cell is the cross-section of an infinite prism, directions are 3-D and
    carried as their projection on the plane; births on the sphere
    (birth_directions), wall entries with the 3-D cosine law
    (wall_births_xy), walks by walk_one_xy; `sampler` must be an x-y one,
    mlp_sampler_xy or walk_sampler_global_xy, and `internal` too,
    mlp_internal_sampler_xy or walk_internal_sampler_xy).
    """
    if geometry not in ("flat", "xy"):
        raise ValueError(geometry)
    walker = walk_one if geometry == "flat" else walk_one_xy
    tau = np.asarray(tau, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    ny, nx = tau.shape
    tf, cf = tau.ravel(), c.ravel()
    flux = np.zeros(ny * nx, dtype=np.float64)
    st = np.zeros(6, dtype=np.float64)
    live = {k: [] for k in ("id", "i", "j", "F", "xi", "gx", "gy", "w", "ev")}
    if wall is not None:
        j, xi, gx, gy = (wall_births if geometry == "flat" else wall_births_xy)(wall, n_hist, seed)
        for h in range(n_hist):
            for k, v in (("id", h), ("i", 0), ("j", int(j[h])), ("F", 3), ("xi", xi[h]),
                         ("gx", gx[h]), ("gy", gy[h]), ("w", 1.0), ("ev", 0)):
                live[k].append(v)
        n_src = 0
    else:
        n_src = n_hist
        srcf = np.maximum(np.asarray(src, dtype=np.float64).ravel(), 0.0)
        cdf = np.cumsum(srcf)
        total = cdf[-1]
        ids = np.arange(n_hist, dtype=np.uint64)
        ub = rng.uniforms_for(seed, ids, np.zeros(n_hist, np.uint32), rng.TAG_BIRTH)
        cells = np.searchsorted(cdf, ub[0] * total, side="left")
        bux, buy = birth_directions(seed, ids, ub[3], geometry)

    # Births: walk from the birth point to the first face crossing (cell frame),
    # or sample that exit with the internal model.
    if internal is not None and n_src > 0:
        face, q, ux, uy, s, ev = internal(ub[1], ub[2], tf[cells], cf[cells], ids, ub[3])
        for h in range(n_hist):
            k = int(cells[h])
            st[3] += 1
            dw, score = deposit(1.0, s[h], tf[k], cf[k])
            flux[k] += score
            st[1] += dw
            w = 1.0 - dw
            w, alive = _roulette(seed, np.array([h], np.uint64), np.array([ev[h]], np.uint32),
                                 np.array([w]), w_cut, p_survive, st)
            if not alive[0]:
                continue
            _advance_one(live, h, k % nx, k // nx, int(face[h]), q[h], ux[h], uy[h], w[0],
                         int(ev[h]), nx, ny, st)
    for h in range(n_src if internal is None else 0):
        k = int(cells[h])
        i, j = k % nx, k // nx
        t, cc = tf[k], cf[k]
        r = walker(t, cc, MODE_IMPLICIT, ub[1, h] * t, ub[2, h] * t, bux[h], buy[h], seed, h, 0)
        st[3] += 1
        st[4] += r["ncoll"]
        dw, score = deposit(1.0, r["s"], t, cc)
        flux[k] += score
        st[1] += dw
        w = 1.0 - dw
        w, alive = _roulette(seed, np.array([h], np.uint64), np.array([r["event"]], np.uint32),
                             np.array([w]), w_cut, p_survive, st)
        if not alive[0]:
            continue
        _advance_one(live, h, i, j, r["face"], r["q"], r["ux"], r["uy"], w[0], r["event"],
                     nx, ny, st)
    L = {k: np.asarray(v) for k, v in live.items()}
    L["id"] = L["id"].astype(np.uint64)
    L["ev"] = L["ev"].astype(np.uint32)
    for L_i in ("i", "j", "F"):
        L[L_i] = L[L_i].astype(np.int64)

    waves = 0
    while L["id"].size > 0:
        waves += 1
        if waves > max_waves:
            raise RuntimeError("too many waves")
        cell = L["j"] * nx + L["i"]
        t, cc = tf[cell], cf[cell]
        rr = np.mod(L["F"] + 1, 4)
        cx, cy = rot(L["gx"], L["gy"], -rr)
        face, q, ux, uy, s, ev = sampler(L["xi"], cx, cy, t, cc, L["id"], L["ev"], rot=rr)
        st[3] += cell.size
        dw, score = deposit(L["w"], s, t, cc)
        np.add.at(flux, cell, score)
        st[1] += dw.sum()
        w = L["w"] - dw
        w, alive = _roulette(seed, L["id"], ev, w, w_cut, p_survive, st)
        G = np.mod(np.asarray(face) + rr, 4)
        gx, gy = rot(ux, uy, rr)
        ni = L["i"] + np.where(G == 1, 1, 0) - np.where(G == 3, 1, 0)
        nj = L["j"] + np.where(G == 2, 1, 0) - np.where(G == 0, 1, 0)
        inside = (ni >= 0) & (ni < nx) & (nj >= 0) & (nj < ny)
        st[0] += w[alive & ~inside].sum()
        keep = alive & inside
        L = {"id": L["id"][keep], "i": ni[keep], "j": nj[keep], "F": np.mod(G[keep] + 2, 4),
             "xi": np.asarray(q)[keep], "gx": gx[keep], "gy": gy[keep], "w": w[keep],
             "ev": np.asarray(ev, np.uint32)[keep]}
    stats = _stats(st)
    stats["waves"] = waves
    return (flux / n_hist).reshape(ny, nx), stats


def _roulette(seed, ids, events, w, w_cut, p_survive, st):
    w = np.asarray(w, dtype=np.float64).copy()
    alive = np.ones(w.shape, dtype=bool)
    low = w < w_cut
    if low.any():
        u = rng.uniforms_for(seed, ids[low], events[low], rng.TAG_ROULETTE)[0]
        surv = u <= p_survive
        wl = w[low]
        st[2] += np.sum(np.where(surv, wl / p_survive - wl, -wl))
        st[5] += np.sum(~surv)
        w[low] = np.where(surv, wl / p_survive, wl)
        alive[np.flatnonzero(low)[~surv]] = False
    return w, alive


def _advance_one(live, h, i, j, G, q, gx, gy, w, ev, nx, ny, st):
    ni = i + (1 if G == 1 else 0) - (1 if G == 3 else 0)
    nj = j + (1 if G == 2 else 0) - (1 if G == 0 else 0)
    if not (0 <= ni < nx and 0 <= nj < ny):
        st[0] += w
        return
    for k, v in (("id", h), ("i", ni), ("j", nj), ("F", (G + 2) % 4), ("xi", q), ("gx", gx),
                 ("gy", gy), ("w", w), ("ev", ev)):
        live[k].append(v)


# ---- rectangular cells in the solve (geometry variant with W != H) --------

def walk_one_rect(tx, ty, c, mode, x, y, ux, uy, seed, pid, event0):
    """One random walk in the rectangle [0, tx] x [0, ty] (optical units) from
    an arbitrary point; q normalized per face. Same outputs as walk_one."""
    status = ctypes.c_int32()
    face = ctypes.c_int32()
    ncoll = ctypes.c_int64()
    ev = ctypes.c_uint32()
    out = np.zeros(6, dtype=np.float64)
    lib().orc_walk_one_rect(float(tx), float(ty), float(c), mode, float(x), float(y), float(ux),
                            float(uy), seed, int(pid), int(event0), ctypes.byref(status),
                            ctypes.byref(face), out.ctypes.data, ctypes.byref(ncoll),
                            ctypes.byref(ev))
    return {"status": status.value, "face": face.value, "q": out[0], "x": out[1], "y": out[2],
            "ux": out[3], "uy": out[4], "s": out[5], "ncoll": ncoll.value, "event": ev.value}


def canonical_sides(tx, ty, rot):
    """Sides of a cell (tx along x, ty along y) in the canonical left-entry
    frame reached by `rot` quarter turns: a quarter turn exchanges them, so
    the canonical width (the depth behind the entry face) is ty and the
    entry face's length tx for odd rot."""
    odd = (np.asarray(rot) % 2) == 1
    return np.where(odd, ty, tx), np.where(odd, tx, ty)


def mlp_sampler_rect(net, steps, integrator, seed):
    """Stage 2 with the network for rectangular cells: condition (xi, cos,
    sin, ln tau_x, c, ln(tau_y / tau_x)) in the canonical frame."""
    def f(xi, cos_c, sin_c, tx_c, ty_c, c, ids, events, rot=None):
        cond = np.stack([xi, cos_c, sin_c, np.log(tx_c), c, np.log(ty_c / tx_c)])
        z = rng.normals_for(seed, ids, events, rng.TAG_NOISE)
        d = mlp.decode(net, mlp.sample(net, cond, z, steps, integrator))
        return d["face"], d["q"], d["ux"], d["uy"], d["s"], np.asarray(events, np.uint32) + 1
    return f


def equivalent_condition_rect(tx, ty, c, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """equivalent_condition for rectangular cells (optical sides tx, ty): the
    implicit-capture walk in the rectangle depends on (c tx, c ty) only, so a
    cell (tx', ty', c') with c' tx' = c tx and c' ty' = c ty has the same
    exits and s = s' c' / c. Both sides must lie in [tau_lo, tau_hi] whatever
    face the particle enters by, so c' is c moved into [c_lo, c_hi] and
    [c max(tx, ty) / tau_hi, c min(tx, ty) / tau_lo]; cells inside the box
    keep (tx, ty, c). Returns (tx', c', ok) with ty' = tx' ty / tx; where no
    equivalent exists (that interval empty, or c = 0) ok is False and the
    cell keeps (tx, c). With tx = ty this is equivalent_condition."""
    tx, ty, c = (np.asarray(a, dtype=np.float64) for a in (tx, ty, c))
    (t_lo, t_hi), (c_lo, c_hi) = tau_range, c_range
    big, small = np.maximum(tx, ty), np.minimum(tx, ty)
    lo = np.maximum(c_lo, c * big / t_hi)
    hi = np.minimum(c_hi, c * small / t_lo)
    ok = (c * small > 0.0) & (lo <= hi)
    inside = ((tx >= t_lo) & (tx <= t_hi) & (ty >= t_lo) & (ty <= t_hi) & (c >= c_lo)
              & (c <= c_hi))
    ok = ok | inside
    cp = np.where(inside, c, np.where(ok, np.clip(c, lo, np.maximum(lo, hi)), c))
    txp = np.where(inside | ~ok, tx, np.clip(c * tx / np.where(ok, cp, 1.0), t_lo, t_hi))
    return txp, cp, ok


def equivalent_sampler_rect(sampler, fallback, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """equivalent_sampler for rectangular cells: each particle sampled by
    `sampler` at its cell's equivalent condition (equivalent_condition_rect,
    in the canonical frame: the interval for c' is the same for either
    orientation) with its track length scaled by c' / c; cells without an
    equivalent go to `fallback` at their own condition."""
    def f(xi, cos_c, sin_c, tx_c, ty_c, c, ids, events, rot=None):
        xi, cos_c, sin_c, tx_c, ty_c, c = (np.asarray(a, dtype=np.float64)
                                           for a in (xi, cos_c, sin_c, tx_c, ty_c, c))
        ids = np.asarray(ids, dtype=np.uint64)
        events = np.asarray(events, dtype=np.uint32)
        txp, cp, ok = equivalent_condition_rect(tx_c, ty_c, c, tau_range, c_range)
        typ = txp * (ty_c / tx_c)
        n = xi.shape[0]
        face = np.zeros(n, np.int64)
        q, ux, uy, s = (np.zeros(n) for _ in range(4))
        ev = np.zeros(n, np.uint32)
        for sel, fn, a, b, cc in ((ok, sampler, txp, typ, cp), (~ok, fallback, tx_c, ty_c, c)):
            k = np.nonzero(sel)[0]
            if k.size == 0:
                continue
            r = None if rot is None else np.asarray(rot)[k]
            fa, qa, uxa, uya, sa, eva = fn(xi[k], cos_c[k], sin_c[k], a[k], b[k], cc[k], ids[k],
                                           events[k], rot=r)
            face[k], q[k], ux[k], uy[k], ev[k] = fa, qa, uxa, uya, eva
            s[k] = np.asarray(sa) * (cc[k] / c[k]) if fn is sampler else sa
        return face, q, ux, uy, s, ev
    return f


def internal_condition_rect(X, Y, tx, ty, c):
    """Condition of the internal model for births in rectangular cells
    (reading of the paper's internal model on the geometry variant with
    W != H): the square model's five components (X, Y, ln tx, c, distance to
    the nearest face in normalized cell units) and the aspect ln(ty / tx),
    the same sixth component as the boundary network's -> [6, B]."""
    X, Y, tx, ty, c = (np.asarray(a, dtype=np.float64) for a in (X, Y, tx, ty, c))
    d = np.minimum(np.minimum(X, Y), np.minimum(1.0 - X, 1.0 - Y))
    return np.stack([X, Y, np.log(tx), c, d, np.log(ty / tx)])


def mlp_internal_sampler_rect(net, steps, integrator, seed):
    """Births in rectangular cells with an internal network of six
    condition components (internal_condition_rect): the exit in the cell's
    own frame from the flow ODE with noise at (id, 0, TAG_NOISE); the next
    event is 1."""
    def f(X, Y, tx, ty, c, ids, u_angle):
        cond = internal_condition_rect(X, Y, tx, ty, c)
        ids = np.asarray(ids, np.uint64)
        z = rng.normals_for(seed, ids, np.zeros(ids.size, np.uint32), rng.TAG_NOISE)
        d = mlp.decode(net, mlp.sample(net, cond, z, steps, integrator))
        return d["face"], d["q"], d["ux"], d["uy"], d["s"], np.ones(ids.size, np.uint32)
    return f


def walk_internal_sampler_rect(seed):
    """Births in rectangular cells walked exactly as the rectangle solve
    walks them: direction on the circle at angle 2 pi u_angle, walk_one_rect
    from (X tx, Y ty) at event 0."""
    def f(X, Y, tx, ty, c, ids, u_angle):
        out = [np.zeros(len(ids)) for _ in range(5)] + [np.zeros(len(ids), np.uint32)]
        for k in range(len(ids)):
            ang = 2.0 * np.pi * u_angle[k]
            r = walk_one_rect(tx[k], ty[k], c[k], MODE_IMPLICIT, X[k] * tx[k], Y[k] * ty[k],
                              np.cos(ang), np.sin(ang), seed, int(ids[k]), 0)
            for a, v in zip(out, (r["face"], r["q"], r["ux"], r["uy"], r["s"], r["event"])):
                a[k] = v
        return out[0].astype(np.int64), out[1], out[2], out[3], out[4], out[5]
    return f


def equivalent_internal_sampler_rect(internal, fallback, tau_range=(0.1, 1000.0),
                                     c_range=(0.5, 0.999)):
    """equivalent_internal_sampler for rectangular cells: births in cells with
    an equivalent condition (equivalent_condition_rect) sampled by `internal`
    at (tx', ty', c') with s scaled by c'/c, the others by `fallback` at their
    own condition."""
    def f(X, Y, tx, ty, c, ids, u_angle):
        X, Y, tx, ty, c = (np.asarray(a, dtype=np.float64) for a in (X, Y, tx, ty, c))
        ids = np.asarray(ids, dtype=np.uint64)
        u_angle = np.asarray(u_angle, dtype=np.float64)
        txp, cp, ok = equivalent_condition_rect(tx, ty, c, tau_range, c_range)
        typ = txp * (ty / tx)
        n = X.shape[0]
        face = np.zeros(n, np.int64)
        q, ux, uy, s = (np.zeros(n) for _ in range(4))
        ev = np.zeros(n, np.uint32)
        for sel, fn, a, b, cc in ((ok, internal, txp, typ, cp), (~ok, fallback, tx, ty, c)):
            k = np.nonzero(sel)[0]
            if k.size == 0:
                continue
            fa, qa, uxa, uya, sa, eva = fn(X[k], Y[k], a[k], b[k], cc[k], ids[k], u_angle[k])
            face[k], q[k], ux[k], uy[k], ev[k] = fa, qa, uxa, uya, eva
            s[k] = np.asarray(sa) * (cc[k] / c[k]) if fn is internal else sa
        return face, q, ux, uy, s, ev
    return f


def internal_pairs_rect(n, seed, tau_range=(0.1, 1000.0), aspect_range=(0.25, 4.0),
                        c_range=(0.5, 0.999)):
    """Training pairs of the internal model for rectangular cells: for
    sample i, the draw (i, 0, tag 11) gives ln tx uniform in the log range, c
    uniform, X and Y uniform; (i, 1, tag 11) the aspect ty / tx log-uniform in
    aspect_range (u0) and the birth direction at angle 2 pi u1 on the circle;
    the implicit-capture walk in the rectangle from (X tx, Y ty) draws from
    event 2. Returns cond [6, n] (internal_condition_rect) and y [4, n] =
    (p, ux, uy, ln s) in the cell's own frame, q normalized per face."""
    ids = np.arange(n, dtype=np.uint64)
    u0 = rng.uniforms_for(seed, ids, np.zeros(n, np.uint32), 11)
    u1 = rng.uniforms_for(seed, ids, np.ones(n, np.uint32), 11)
    lo, hi = np.log(tau_range[0]), np.log(tau_range[1])
    tx = np.exp(lo + (hi - lo) * u0[0])
    c = c_range[0] + (c_range[1] - c_range[0]) * u0[1]
    X, Y = u0[2], u0[3]
    alo, ahi = np.log(aspect_range[0]), np.log(aspect_range[1])
    ty = tx * np.exp(alo + (ahi - alo) * u1[0])
    ang = 2.0 * np.pi * u1[1]
    y = np.zeros((4, n))
    for i in range(n):
        w = walk_one_rect(tx[i], ty[i], c[i], MODE_IMPLICIT, X[i] * tx[i], Y[i] * ty[i],
                          np.cos(ang[i]), np.sin(ang[i]), seed, i, 2)
        y[:, i] = (w["face"] + w["q"], w["ux"], w["uy"], np.log(max(w["s"], mlp.S_MIN)))
    return internal_condition_rect(X, Y, tx, ty, c), y


def walk_sampler_rect(seed):
    """Stage 2 replaced by the implicit-capture walk in the canonical frame of
    a rectangular cell, as the training pairs take it (transmit_rect: entry
    on the left face at y = xi ty_c, width tx_c behind it): the solve with
    this sampler reproduces a random-walk solve only if the canonical sides
    the solve hands over match the convention of the training pairs."""
    def f(xi, cos_c, sin_c, tx_c, ty_c, c, ids, events, rot=None):
        r = transmit_rect(xi, cos_c, sin_c, tx_c, ty_c, c, MODE_IMPLICIT, seed, ids=ids,
                          events=events)
        return r["face"], r["q"], r["ux"], r["uy"], r["s"], r["events"]
    return f


def walk_sampler_global_rect(seed):
    """The random walk through a rectangular cell in the cell's own (global)
    frame, as a random-walk solve takes it (walk_sampler_global for
    rectangles): entry face F = (rot - 1) mod 4 at counter-clockwise
    parameter 1 - xi, the exit returned in the canonical frame."""
    def f(xi, cos_c, sin_c, tx_c, ty_c, c, ids, events, rot=None):
        n = len(ids)
        face = np.zeros(n, np.int64)
        out = [np.zeros(n) for _ in range(4)]
        ev = np.zeros(n, np.uint32)
        for k in range(n):
            r = int(rot[k])
            tx, ty = (ty_c[k], tx_c[k]) if r % 2 else (tx_c[k], ty_c[k])  # global sides
            F = (r - 1) % 4
            x = float(xi[k])
            X, Y = {0: (1.0 - x, 0.0), 1: (1.0, 1.0 - x), 2: (x, 1.0), 3: (0.0, x)}[F]
            gx, gy = rot_dir(cos_c[k], sin_c[k], r)
            w = walk_one_rect(tx, ty, c[k], MODE_IMPLICIT, X * tx, Y * ty, gx, gy, seed,
                              int(ids[k]), int(events[k]))
            face[k] = (w["face"] - r) % 4
            ux, uy = rot_dir(w["ux"], w["uy"], -r)
            out[0][k], out[1][k], out[2][k], out[3][k] = w["q"], ux, uy, w["s"]
            ev[k] = w["event"]
        return face, out[0], out[1], out[2], out[3], ev
    return f


def solve_gmc_rect(sigma, c, src, dx, dy, n_hist, seed, sampler, w_cut=1e-4, p_survive=0.1,
                   max_waves=100000, wall=None, internal=None):
    """The event-based solve on a grid of rectangular cells of physical size
    dx x dy (every cell alike) with cross sections sigma [ny, nx] and
    scattering ratios c: cell (i, j) has optical sides tx = sigma dx (along x)
    and ty = sigma dy. Births as solve_gmc (cell by the source CDF, point
    (X tx, Y ty), direction on the circle), walked with walk_one_rect; every
    later crossing goes to `sampler` in the canonical frame with the
    canonical sides (canonical_sides). Flux per source particle per unit
    area: Delta w / (sigma_a dx dy) per Eq. 7 (the track length w l / (dx dy)
    for c = 1). Returns (flux [ny, nx], stats). With dx = dy = 1 this is
    solve_gmc on tau = sigma.
    wall: [ny] strengths of a surface source on the left boundary instead of
    src (wall_births: row by strength, uniform height on the boundary cell's
    left face, the cosine law; weight 1, next event 0); its first crossing
    goes to `sampler` like every later one.
    internal: sampler of births (mlp_internal_sampler_rect,
    walk_internal_sampler_rect) called as internal(X, Y, tx, ty, c, ids,
    u_angle), or None to walk every birth."""
    sig = np.asarray(sigma, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    ny, nx = sig.shape
    sf, cf = sig.ravel(), c.ravel()
    txf, tyf = sf * dx, sf * dy
    area = float(dx) * float(dy)
    flux = np.zeros(ny * nx, dtype=np.float64)
    st = np.zeros(6, dtype=np.float64)
    live = {k: [] for k in ("id", "i", "j", "F", "xi", "gx", "gy", "w", "ev")}
    n_src = n_hist
    if wall is not None:
        j, xi, gx, gy = wall_births(wall, n_hist, seed)
        for h in range(n_hist):
            for k, v in (("id", h), ("i", 0), ("j", int(j[h])), ("F", 3), ("xi", xi[h]),
                         ("gx", gx[h]), ("gy", gy[h]), ("w", 1.0), ("ev", 0)):
                live[k].append(v)
        n_src = 0
    else:
        srcf = np.maximum(np.asarray(src, dtype=np.float64).ravel(), 0.0)
        cdf = np.cumsum(srcf)
        ids = np.arange(n_hist, dtype=np.uint64)
        ub = rng.uniforms_for(seed, ids, np.zeros(n_hist, np.uint32), rng.TAG_BIRTH)
        cells = np.searchsorted(cdf, ub[0] * cdf[-1], side="left")
        bux, buy = birth_directions(seed, ids, ub[3], "flat")
    if internal is not None and n_src > 0:
        bf, bq, bux_, buy_, bs, bev = internal(ub[1], ub[2], txf[cells], tyf[cells], cf[cells], ids,
                                               ub[3])
    for h in range(n_src):
        k = int(cells[h])
        if internal is not None:
            r = {"face": int(bf[h]), "q": bq[h], "ux": bux_[h], "uy": buy_[h], "s": bs[h],
                 "event": int(bev[h]), "ncoll": 0}
        else:
            r = walk_one_rect(txf[k], tyf[k], cf[k], MODE_IMPLICIT, ub[1, h] * txf[k],
                              ub[2, h] * tyf[k], bux[h], buy[h], seed, h, 0)
        st[3] += 1
        st[4] += r["ncoll"]
        dw, score = deposit(1.0, r["s"], sf[k], cf[k])
        flux[k] += score / area
        st[1] += dw
        w, alive = _roulette(seed, np.array([h], np.uint64), np.array([r["event"]], np.uint32),
                             np.array([1.0 - dw]), w_cut, p_survive, st)
        if alive[0]:
            _advance_one(live, h, k % nx, k // nx, r["face"], r["q"], r["ux"], r["uy"], w[0],
                         r["event"], nx, ny, st)
    L = {k: np.asarray(v) for k, v in live.items()}
    L["id"] = L["id"].astype(np.uint64)
    L["ev"] = L["ev"].astype(np.uint32)
    for key in ("i", "j", "F"):
        L[key] = L[key].astype(np.int64)
    waves = 0
    while L["id"].size > 0:
        waves += 1
        if waves > max_waves:
            raise RuntimeError("too many waves")
        cell = L["j"] * nx + L["i"]
        rr = np.mod(L["F"] + 1, 4)
        cx, cy = rot(L["gx"], L["gy"], -rr)
        txc, tyc = canonical_sides(txf[cell], tyf[cell], rr)
        face, q, ux, uy, s, ev = sampler(L["xi"], cx, cy, txc, tyc, cf[cell], L["id"], L["ev"],
                                         rot=rr)
        st[3] += cell.size
        dw, score = deposit(L["w"], s, sf[cell], cf[cell])
        np.add.at(flux, cell, score / area)
        st[1] += dw.sum()
        w, alive = _roulette(seed, L["id"], ev, L["w"] - dw, w_cut, p_survive, st)
        G = np.mod(np.asarray(face) + rr, 4)
        gx, gy = rot(ux, uy, rr)
        ni = L["i"] + np.where(G == 1, 1, 0) - np.where(G == 3, 1, 0)
        nj = L["j"] + np.where(G == 2, 1, 0) - np.where(G == 0, 1, 0)
        inside = (ni >= 0) & (ni < nx) & (nj >= 0) & (nj < ny)
        st[0] += w[alive & ~inside].sum()
        keep = alive & inside
        L = {"id": L["id"][keep], "i": ni[keep], "j": nj[keep], "F": np.mod(G[keep] + 2, 4),
             "xi": np.asarray(q)[keep], "gx": gx[keep], "gy": gy[keep], "w": w[keep],
             "ev": np.asarray(ev, np.uint32)[keep]}
    stats = _stats(st)
    stats["waves"] = waves
    return (flux / n_hist).reshape(ny, nx), stats
