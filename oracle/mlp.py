"""Oracle: the GMC velocity network and flow-ODE sampler in FP64 (test
infrastructure only).

What it computes, in the paper's order:
  * Eq. 8 -- a sample is x(1) of dx/dt = v_theta(x, t), x(0) ~ N(0, I),
    integrated from t = 0 to 1 with a fixed number of steps (explicit Euler,
    the explicit midpoint rule, or classical RK4, which the paper times).
  * Eq. 10 / Eq. 11 -- the condition c is the entry state and cell in optical
    coordinates and the state x is the exit state y = (p_exit, Omega_exit, s).
    Here the cell is a square and directions lie on the unit circle, so
    c = (xi_in, cos theta_in, sin theta_in, ln tau, c_scat) and
    y = (p, cos theta_out, sin theta_out, ln s).
  * v_theta is a plain feed-forward network: input [c_std (5), x (4),
    emb(t) (16)], four hidden layers of width 256 with SiLU, linear output 4.
    emb(t) = [sin(2^j pi t)]_{j<8} followed by [cos(2^j pi t)]_{j<8}.
  * The residual-modulated network is this build's reading of the paper's
    own architecture (section "Network Architecture and Inputs": residual
    blocks with adaptive modulation conditioned on the physical context; its
    specification is in a supplement that is not available). Layer 1 is as
    above (t and c enter through its learned columns); layers 2-4 become
    residual blocks whose pre-activation is shifted by a learned linear map
    of the condition and scaled channel-wise by the cell's optical
    properties (standardized ln tau and c, condition components 3 and 4):
        z_l = W_l a_{l-1} + b_l + M_l c_std
        g_l = 1 + G_l[0] c_std[3] + G_l[1] c_std[4]
        a_l = a_{l-1} + SiLU(g_l * z_l)            (l = 2, 3, 4)
    and v = W_5 a_4 + b_5. M_l is [256][5], G_l is [2][256]; with G = 0 and
    M = 0 it is a plain residual network.
  * Rectangular cells (the condition of the section "Network Architecture
    and Inputs" with W != H): a sixth condition component, ln(tau_y / tau_x)
    for a cell of optical width tau_x (the depth, along the entry direction's
    normal) and height tau_y (the entry face), after ln tau_x and c; it
    enters the network as input column 25, after the time embedding, so the
    first 25 columns keep the square network's meaning (a square cell has
    aspect 0). Weight files of such networks have n_cond = 6 and 26 inputs.
  * Decoding (the fourth stage of the transport algorithm): destandardize,
    wrap p into [0,4), split it into face and position, renormalize the
    direction, make it point out of the exit face, s = exp(ln s).
    decode_disk is the decoding of x-y geometry, whose directions are 3-D and
    enter the network by their projection on the unit disk: the projection
    is pulled back into the disk instead of onto the circle.

Matrix products use numpy's matmul in float64 (a library primitive); nothing
is blocked, fused or reordered beyond the definitions above.

The paper fixes no reduced precision. For an 8-bit path this module also
defines the quantized network such a path evaluates (quantized_e4m3): the
three 256 x 256 layers take E4M3 weights with one FP32 scale per output row
(s_c = max_k |W[c,k]| / 448) and E4M3 inputs with unit scale; everything
else stays as above, in FP64. It is the same network up to those roundings,
so the FP64 results stay the reference for the size of the 8-bit error.

Weight file ("GMCW" version 1, little-endian):
  char magic[4] = "GMCW"; u32 version; u32 n_layers = 5; u32 dims[6];
  u32 n_cond, n_state, n_emb, flags;
  f32 cond_mean[n_cond], cond_std[n_cond], y_mean[4], y_std[4];
  (n_cond = 5 with dims[0] = 25, or 6 with dims[0] = 26 for rectangular cells)
  then per layer l: f32 W_l[dims[l+1]][dims[l]] (out x in), f32 b_l[dims[l+1]].
  flags bit 0 marks the residual-modulated network, whose file continues
  with f32 M[3][256][5] (layers 2-4) and f32 G[3][2][256].
"""
import struct

import numpy as np

N_COND = 5
N_STATE = 4
N_EMB = 16
HIDDEN = 256
DIMS = (N_COND + N_STATE + N_EMB, HIDDEN, HIDDEN, HIDDEN, HIDDEN, N_STATE)
S_MIN = 1e-7
FLAG_RM = 1  # weight-file flag of the residual-modulated network


class Net:
    """FP64 copy of a weight file: W[l] (out x in), b[l], standardization;
    for the residual-modulated network also M[j] ([256][5]) and G[j]
    ([2][256]) of hidden layer j + 2 (rm is True)."""

    def __init__(self, W, b, cond_mean, cond_std, y_mean, y_std, M=None, G=None):
        self.W = [np.asarray(w, dtype=np.float64) for w in W]
        self.b = [np.asarray(v, dtype=np.float64) for v in b]
        self.cond_mean = np.asarray(cond_mean, dtype=np.float64)
        self.cond_std = np.asarray(cond_std, dtype=np.float64)
        self.y_mean = np.asarray(y_mean, dtype=np.float64)
        self.y_std = np.asarray(y_std, dtype=np.float64)
        self.rm = M is not None
        if self.rm:
            self.M = [np.asarray(m, dtype=np.float64).reshape(HIDDEN, N_COND) for m in M]
            self.G = [np.asarray(q, dtype=np.float64).reshape(2, HIDDEN) for q in G]


def read_weights(path):
    with open(path, "rb") as f:
        blob = f.read()
    if blob[:4] != b"GMCW":
        raise ValueError("not a GMCW weight file")
    version, n_layers = struct.unpack_from("<2I", blob, 4)
    dims = struct.unpack_from("<6I", blob, 12)
    n_cond, n_state, n_emb, flags = struct.unpack_from("<4I", blob, 36)
    if (version != 1 or n_layers != 5 or n_cond not in (N_COND, N_COND + 1)
            or tuple(dims) != (n_cond + N_STATE + N_EMB,) + DIMS[1:]
            or (n_state, n_emb) != (N_STATE, N_EMB) or flags & ~FLAG_RM
            or (n_cond != N_COND and flags & FLAG_RM)):
        raise ValueError("unsupported weight file layout")
    off = 52
    ns = 2 * n_cond + 2 * N_STATE
    stats = np.frombuffer(blob, dtype="<f4", count=ns, offset=off).astype(np.float64)
    off += ns * 4
    W, b = [], []
    for l in range(5):
        n_out, n_in = dims[l + 1], dims[l]
        W.append(np.frombuffer(blob, dtype="<f4", count=n_out * n_in, offset=off)
                 .reshape(n_out, n_in).astype(np.float64))
        off += n_out * n_in * 4
        b.append(np.frombuffer(blob, dtype="<f4", count=n_out, offset=off).astype(np.float64))
        off += n_out * 4
    M = G = None
    if flags & FLAG_RM:
        M, G = [], []
        for _ in range(3):
            M.append(np.frombuffer(blob, dtype="<f4", count=HIDDEN * N_COND, offset=off)
                     .reshape(HIDDEN, N_COND).astype(np.float64))
            off += HIDDEN * N_COND * 4
        for _ in range(3):
            G.append(np.frombuffer(blob, dtype="<f4", count=2 * HIDDEN, offset=off)
                     .reshape(2, HIDDEN).astype(np.float64))
            off += 2 * HIDDEN * 4
    if off != len(blob):
        raise ValueError("weight file has trailing or missing bytes")
    k = n_cond
    return Net(W, b, stats[0:k], stats[k:2 * k], stats[2 * k:2 * k + 4], stats[2 * k + 4:2 * k + 8],
               M, G)


def time_embedding(t):
    """emb(t) for t of shape [B] -> [B, 16]."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    freq = (2.0 ** np.arange(8)) * np.pi
    ang = t[:, None] * freq[None, :]
    return np.concatenate([np.sin(ang), np.cos(ang)], axis=1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def standardize_cond(net, cond):
    """cond: [n_cond, B] raw features -> [B, n_cond] standardized."""
    cond = np.asarray(cond, dtype=np.float64)
    return ((cond.T - net.cond_mean) / net.cond_std)


def round_e4m3(a):
    """Nearest value of the FP8 E4M3 format, ties to an even significand,
    saturating at +-448.

    E4M3 (OCP 8-bit floating point): sign, 4 exponent bits with bias 7, 3
    significand bits, no infinities. Normal values (1 + m/8) 2^(e-7) for
    e = 1..15 (e = 15, m = 7 is NaN, so 448 = 1.75 * 2^8 is the largest);
    subnormal values m/8 * 2^-6. In the binade [2^E, 2^(E+1)) the spacing is
    2^(E-3); below 2^-6 it is 2^-9.
    """
    a = np.asarray(a, dtype=np.float64)
    m = np.minimum(np.abs(a), 448.0)
    _, ex = np.frexp(np.maximum(m, 2.0 ** -6))  # m = f 2^ex with f in [0.5, 1)
    q = np.ldexp(1.0, ex - 1 - 3)                # spacing in m's binade
    r = np.round(m / q) * q                       # numpy rounds halves to even
    return np.copysign(np.minimum(r, 448.0), a)


def quantized_e4m3(net):
    """The network an E4M3 path evaluates (see the module note): W2..W4 rows
    replaced by s_c round_e4m3(W[c,:] / s_c) with s_c = max_k |W[c,k]| / 448
    (1 for an all-zero row), and the inputs of those layers rounded to E4M3.
    """
    if getattr(net, "rm", False):
        raise ValueError("the E4M3 network is defined for the plain MLP only")
    W = [w.copy() for w in net.W]
    for l in (1, 2, 3):
        amax = np.abs(W[l]).max(axis=1)
        sc = np.where(amax > 0, amax / 448.0, 1.0)[:, None]
        W[l] = round_e4m3(W[l] / sc) * sc
    q = Net(W, net.b, net.cond_mean, net.cond_std, net.y_mean, net.y_std)
    q.e4m3_inputs = True
    return q


def network_input(cn, x, t):
    """Layer-1 input [cn(5), x(4), emb(t)(16)] and, for rectangular cells
    (cn with 6 columns), the aspect component as column 25."""
    return np.concatenate([cn[:, :N_COND], x, time_embedding(t), cn[:, N_COND:]], axis=1)


def velocity(net, cn, x, t):
    """v_theta(x, t | c): cn [B,5] (or [B,6] for rectangular cells)
    standardized condition, x [B,4], t scalar or [B]."""
    B = x.shape[0]
    t = np.broadcast_to(np.asarray(t, dtype=np.float64), (B,))
    h = network_input(cn, x, t)
    if getattr(net, "rm", False):
        return velocity_rm(net, cn, h)
    e4m3 = getattr(net, "e4m3_inputs", False)
    for l in range(4):
        if e4m3 and l >= 1:
            h = round_e4m3(h)
        h = silu(h @ net.W[l].T + net.b[l])
    return h @ net.W[4].T + net.b[4]


def velocity_rm(net, cn, h):
    """The residual-modulated network (module note) on layer-1 inputs h
    [B, 25] with standardized conditions cn [B, 5]."""
    a = silu(h @ net.W[0].T + net.b[0])
    for j in range(3):
        z = a @ net.W[j + 1].T + net.b[j + 1] + cn @ net.M[j].T
        g = 1.0 + cn[:, 3:4] * net.G[j][0][None, :] + cn[:, 4:5] * net.G[j][1][None, :]
        a = a + silu(g * z)
    return a @ net.W[4].T + net.b[4]


def integrate(vfun, x0, steps, integrator="euler"):
    """Fixed-step integration of dx/dt = vfun(x, t) from t = 0 to 1.

    Euler:    x_{k+1} = x_k + h v(x_k, t_k)
    midpoint: x_{k+1} = x_k + h v(x_k + (h/2) v(x_k, t_k), t_k + h/2)
    rk4:      k1 = v(x_k, t_k), k2 = v(x_k + (h/2) k1, t_k + h/2),
              k3 = v(x_k + (h/2) k2, t_k + h/2), k4 = v(x_k + h k3, t_k + h),
              x_{k+1} = x_k + (h/6)(k1 + 2 k2 + 2 k3 + k4)   (classical Runge-Kutta,
              the fixed-step solver the paper times)
    with h = 1/steps and t_k = k h.
    """
    x = np.array(x0, dtype=np.float64)
    h = 1.0 / steps
    for k in range(steps):
        t = k * h
        if integrator == "euler":
            x = x + h * vfun(x, t)
        elif integrator == "midpoint":
            xm = x + 0.5 * h * vfun(x, t)
            x = x + h * vfun(xm, t + 0.5 * h)
        elif integrator == "rk4":
            k1 = vfun(x, t)
            k2 = vfun(x + 0.5 * h * k1, t + 0.5 * h)
            k3 = vfun(x + 0.5 * h * k2, t + 0.5 * h)
            k4 = vfun(x + h * k3, t + h)
            x = x + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        else:
            raise ValueError(integrator)
    return x


def sample(net, cond, noise, steps, integrator="euler"):
    """Eq. 8: x(1) from x(0) = noise ([4, B]) for raw conditions cond ([5, B]).

    Returns the standardized x(1) as [4, B].
    """
    cn = standardize_cond(net, cond)
    x0 = np.asarray(noise, dtype=np.float64).T
    return integrate(lambda x, t: velocity(net, cn, x, t), x0, steps, integrator).T


OUTWARD = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])


def decode(net, y_raw):
    """Standardized ODE output [4, B] -> exit state dict (canonical frame).

    face in {0 bottom, 1 right, 2 top, 3 left}, q the counter-clockwise
    position on that face, (ux, uy) a unit direction pointing out of the face,
    s the track length in optical units (at least S_MIN).
    """
    y = np.asarray(y_raw, dtype=np.float64).T * net.y_std + net.y_mean
    p = np.mod(y[:, 0], 4.0)
    face = np.minimum(np.floor(p), 3.0).astype(np.int64)
    q = np.clip(p - face, 0.0, 1.0)
    ux, uy = y[:, 1].copy(), y[:, 2].copy()
    norm = np.hypot(ux, uy)
    n_out = OUTWARD[face]
    zero = norm == 0.0
    ux = np.where(zero, n_out[:, 0], ux / np.where(zero, 1.0, norm))
    uy = np.where(zero, n_out[:, 1], uy / np.where(zero, 1.0, norm))
    dot = ux * n_out[:, 0] + uy * n_out[:, 1]
    inward = dot < 0.0
    ux = np.where(inward, ux - 2.0 * dot * n_out[:, 0], ux)
    uy = np.where(inward, uy - 2.0 * dot * n_out[:, 1], uy)
    s = np.maximum(np.exp(y[:, 3]), S_MIN)
    return {"face": face, "q": q, "ux": ux, "uy": uy, "s": s, "inward": inward}


def decode_disk(net, y_raw):
    """Standardized ODE output [4, B] -> exit state for x-y geometry, where
    (y1, y2) is the projection of a 3-D unit direction on the unit disk.

    face, q and s as in decode; the projection is scaled back onto the unit
    circle when it falls outside the disk, its component along the exit
    face's normal is reflected when it points inward, and one with no outward
    component left (parallel to the face, or zero) becomes the outward
    normal. uz is the out-of-plane magnitude sqrt(1 - ux^2 - uy^2) (its sign
    does not enter a walk in the plane).
    """
    y = np.asarray(y_raw, dtype=np.float64).T * net.y_std + net.y_mean
    p = np.mod(y[:, 0], 4.0)
    face = np.minimum(np.floor(p), 3.0).astype(np.int64)
    q = np.clip(p - face, 0.0, 1.0)
    ux, uy = y[:, 1].copy(), y[:, 2].copy()
    norm = np.hypot(ux, uy)
    big = norm > 1.0
    ux = np.where(big, ux / np.where(big, norm, 1.0), ux)
    uy = np.where(big, uy / np.where(big, norm, 1.0), uy)
    n_out = OUTWARD[face]
    dot = ux * n_out[:, 0] + uy * n_out[:, 1]
    inward = dot < 0.0
    ux = np.where(inward, ux - 2.0 * dot * n_out[:, 0], ux)
    uy = np.where(inward, uy - 2.0 * dot * n_out[:, 1], uy)
    flat = dot == 0.0
    ux = np.where(flat, n_out[:, 0], ux)
    uy = np.where(flat, n_out[:, 1], uy)
    uz = np.sqrt(np.maximum(1.0 - ux * ux - uy * uy, 0.0))
    s = np.maximum(np.exp(y[:, 3]), S_MIN)
    return {"face": face, "q": q, "ux": ux, "uy": uy, "uz": uz, "s": s, "inward": inward}
