"""Plain FP64 CPU oracle for sp-DBA (spectral dynamic block activation).

TEST INFRASTRUCTURE ONLY: used by tests/, by the smoke check and by the
benchmark's CPU-baseline and reference legs.  The CUDA path never imports it.

Every function follows the paper's description step by step, in FP64, with
numpy for elementwise arithmetic and the oracle's own C FFT
(oracle_fft.c) for transforms.  Nothing is fused or reordered beyond what the
cited passage states.

Parity status of each piece (what pins it, see tests/test_oracle_*.py):
  fftn / ifftn ................ brute-force DFT, Parseval, round trip
  ch_regular_step ............. single-mode closed-form growth factor, k=0 conservation
  block_measures / classify ... hand-built block maps with known dilations
  sigma_field ................. closed form of the taper product (Eq. S.2, S.3)
  masked steps ................ threshold 0 == Regular bit for bit; infinite threshold
                                leaves every block but the k=0 block untouched
  threshold_control /
  ThresholdController ......... hand-traced threshold sequences on synthetic ratio
                                histories (every branch and both deadband edges);
                                control steps are full-activation steps (== Regular)
  nls_* ....................... CW exact solution, dispersion-only closed form,
                                unitarity, forward/backward recovery
  half-spectrum form (*_half) . numpy's rfftn / irfftn (incl. a stored kx = 0 plane that
                                is not conjugate-symmetric), Eq. S.4 extension == full DFT,
                                Regular half step == half of the full Regular step,
                                hand-traced half maps (conjugate neighbours across kx = 0
                                and past the Nyquist block) and their sigma, threshold 0 ==
                                Regular bit for bit, untouched frozen modes
  rcd_* ....................... circulant eigenvalues in closed form, hand-computed
                                reaction values, direct solve == eigen form,
                                linearised single-mode growth matrix, threshold 0 ==
                                Regular bit for bit
No function here is "parity unpinned".

Paper conventions restated (section / equation of arXiv 2609.03922):
  * Block partition of the transformed field into fixed B^d blocks (Methods,
    "Spectral dynamic block activation").
  * States: ACTIVE when the block's activation measure meets the threshold;
    TRANSITION when not active but a neighbouring block is active; FROZEN
    otherwise (Methods).
  * Real fields may be stored as the half spectrum kx = 0 .. N/2 with the block map
    on that half; a neighbour in the omitted half is activated through its
    conjugate counterpart, X(-k) = conj X(k), and kx = 0 is a symmetry boundary
    (S1.2, Eq. S.4).
  * Transition smoothing q_{n+1} = q_n + sigma(k) dq_raw with the taper
    w(i) = (1 - cos(pi i / (B-1))) / 2 and sigma the product of w over the
    faces whose neighbour is frozen (S1.1, Eq. S.1-S.3).
  * The block holding the zero-frequency mode is kept active (S6.1).
  * Periodic refresh activates every block every F steps (S1.3); a warm-up of
    all-active steps precedes adaptive operation (S3.2).
  * Dynamic threshold control (S1.3): every control interval the measured
    mean share r of non-frozen (active + transition) blocks is compared with
    a target r_tar; outside the relative deadband eta the threshold is scaled
    by 1 + eta or 1 - eta, and by 2 or 1/2 when r / r_tar > 2 or < 0.5; each
    check is followed by one full-activation step (S1.3, S3.2 parameters).
  * Semi-implicit Fourier update of a conserved (Cahn-Hilliard form) field
    (S3.1 dynamics, S4.2 semi-implicit update with M = 1).
  * Reaction-cross-diffusion (S4.1-S4.3): M components, symmetric circulant
    cross-diffusion matrix D, generalised Lotka-Volterra reaction evaluated in
    real space, semi-implicit update (I + dt k^2 D)^{-1}[u + dt R] per mode,
    directly or through D = V Lambda V^T; activation by the component RMS
    Fourier amplitude, one state per block for all M components.
  * Symmetric split-step Fourier with the linear operator applied in two
    frequency-domain half-steps and the Kerr phase in the time domain (S5.1,
    S5.2); recovery metrics NMSE and field correlation (S5.3).
"""
import ctypes
import math

import numpy as np

from . import build_oracle

STATE_FROZEN = 0
STATE_TRANSITION = 1
STATE_ACTIVE = 2

MEASURE_MAXAMP = 0   # A_B = max_{k in B} |q(k)|              (S4.2 any-mode amplitude)
MEASURE_ENERGY = 1   # ||q_B||_2 = sqrt(sum_{k in B} |q(k)|^2)  (Results 2.1 block energy)

TAU_REL_MAX = 0      # tau = threshold * max |q(k)|  (k = 0 excluded for the conserved CH field)
TAU_ABS = 1          # tau = threshold

__all__ = [
    "STATE_FROZEN", "STATE_TRANSITION", "STATE_ACTIVE", "MEASURE_MAXAMP", "MEASURE_ENERGY",
    "TAU_REL_MAX", "TAU_ABS", "fftn", "ifftn", "fft_batch", "ifft_batch", "num_threads",
    "wavenumbers", "k_squared", "taper", "block_counts", "block_measures", "global_max_sq",
    "threshold_value", "classify", "sigma_field", "ch_regular_step", "ch_masked_step",
    "ch_real_field", "ch_mass", "CHConfig", "run_ch", "nls_omega", "nls_half_factor",
    "nls_kerr", "nls_masked_half", "nls_regular_step", "nls_masked_step", "NLSConfig",
    "run_nls", "rel_l2", "nmse_db", "field_corr", "assess_states", "effective_states",
    "threshold_control", "ThresholdController", "is_control_step",
    "rcd_diffusion_matrix", "rcd_interaction_matrix", "rcd_reaction", "rcd_homogeneous_state",
    "rcd_eigen", "rcd_update_direct", "rcd_update_eigen", "rcd_mode_amplitude_sq", "RCDConfig",
    "rcd_assess_states", "rcd_real_field", "rcd_new", "rcd_masked_step", "run_rcd",
    "half_extent", "rfftn_half", "hermitian_extend", "ch_real_field_half", "half_block_counts",
    "half_block_measures", "half_neighbour", "classify_half", "sigma_field_half", "k_squared_half",
    "ch_regular_step_half", "ch_masked_step_half", "assess_states_half", "run_ch_half",
]

# --------------------------------------------------------------------------------------
# FFT (the oracle's own C implementation)
# --------------------------------------------------------------------------------------
_lib = None


def _load():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        lib = ctypes.CDLL(path)
        lib.oracle_fftn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_long),
                                    ctypes.c_int, ctypes.c_int]
        lib.oracle_fftn.restype = ctypes.c_int
        lib.oracle_fft1_batch.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_long,
                                          ctypes.c_int, ctypes.c_int]
        lib.oracle_fft1_batch.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle's FFT uses."""
    return int(_load().oracle_num_threads())


def _fftn(x, sign, normalize):
    a = np.array(x, dtype=np.complex128, order="C", copy=True)
    dims = (ctypes.c_long * a.ndim)(*a.shape)
    rc = _load().oracle_fftn(a.ctypes.data, a.ndim, dims, sign, 1 if normalize else 0)
    if rc != 0:
        raise RuntimeError("oracle_fftn failed (%d)" % rc)
    return a


def fftn(x):
    """Forward DFT over every axis: X[k] = sum_n x[n] exp(-2 pi i n.k / N)."""
    return _fftn(x, -1, False)


def ifftn(x):
    """Inverse DFT over every axis with the 1/N normalisation."""
    return _fftn(x, +1, True)


def _fft_batch(x, sign, normalize):
    a = np.array(x, dtype=np.complex128, order="C", copy=True)
    if a.ndim != 2:
        raise ValueError("expected (batch, n)")
    rc = _load().oracle_fft1_batch(a.ctypes.data, a.shape[0], a.shape[1], sign,
                                   1 if normalize else 0)
    if rc != 0:
        raise RuntimeError("oracle_fft1_batch failed (%d)" % rc)
    return a


def fft_batch(x):
    """Forward 1-D DFT of each row of a (batch, n) array."""
    return _fft_batch(x, -1, False)


def ifft_batch(x):
    """Inverse 1-D DFT (with 1/n) of each row of a (batch, n) array."""
    return _fft_batch(x, +1, True)


# --------------------------------------------------------------------------------------
# Grids, blocks and block states
# --------------------------------------------------------------------------------------
def wavenumbers(n, dx=1.0):
    """Angular wavenumbers of a periodic axis in FFT order: 2 pi j/(n dx) for j <= n/2,
    2 pi (j - n)/(n dx) above."""
    j = np.arange(n, dtype=np.float64)
    j = np.where(j <= n // 2, j, j - n)
    return 2.0 * math.pi * j / (n * dx)


def k_squared(dims, dx=1.0):
    """|k|^2 on the full (complex) spectral grid, same shape as the field."""
    k2 = np.zeros(tuple(dims), dtype=np.float64)
    for axis, n in enumerate(dims):
        shape = [1] * len(dims)
        shape[axis] = n
        k2 = k2 + wavenumbers(n, dx).reshape(shape) ** 2
    return k2


def taper(B):
    """1-D transition taper w(i) = (1 - cos(pi i / (B-1))) / 2, i = 0..B-1 (S1.1, Eq. S.2)."""
    if B < 2:
        return np.ones(B)
    i = np.arange(B, dtype=np.float64)
    return 0.5 * (1.0 - np.cos(math.pi * i / (B - 1)))


def block_counts(dims, block):
    for n, b in zip(dims, block):
        if b < 1 or n % b != 0:
            raise ValueError("block edge %d does not divide %d" % (b, n))
    return tuple(n // b for n, b in zip(dims, block))


def _blockify(a, block):
    """View a field of shape dims as (nb0, B0, nb1, B1, ...)."""
    nbs = block_counts(a.shape, block)
    shape = []
    for nb, b in zip(nbs, block):
        shape += [nb, b]
    return a.reshape(shape)


def _mode_sq(q):
    """|q|^2 = re^2 + im^2 in FP64 (re^2 and im^2 rounded separately, then added)."""
    re = np.real(q).astype(np.float64)
    im = np.imag(q).astype(np.float64)
    return re * re + im * im


def block_measures(q, block):
    """Per-block max |q|^2 and sum |q|^2 (FP64), shape = block grid."""
    sq = _blockify(_mode_sq(q), block)
    axes = tuple(range(1, sq.ndim, 2))
    return sq.max(axis=axes), sq.sum(axis=axes)


def global_max_sq(q, exclude_dc):
    """max |q(k)|^2 over the whole field, optionally excluding k = 0."""
    sq = _mode_sq(q)
    if exclude_dc:
        sq = sq.copy()
        sq.flat[0] = 0.0
    return float(sq.max())


def threshold_value(q, threshold, tau_rule, exclude_dc):
    """tau = threshold * max |q(k)| (REL_MAX) or tau = threshold (ABS)."""
    if tau_rule == TAU_ABS:
        return float(threshold)
    return float(threshold) * math.sqrt(global_max_sq(q, exclude_dc))


def classify(measure, tau, force_dc=False, transitions=True):
    """Block states from per-block measures (Methods; S1.1).

    ACTIVE iff measure >= tau; the block holding k = 0 is forced ACTIVE when
    force_dc (S6.1).  With transitions, a non-active block with an ACTIVE face
    neighbour (periodic wrap of the block index) is TRANSITION; the rest are
    FROZEN.
    """
    active = np.asarray(measure, dtype=np.float64) >= tau
    if force_dc:
        active.flat[0] = True
    states = np.where(active, STATE_ACTIVE, STATE_FROZEN).astype(np.uint8)
    if transitions:
        near = np.zeros_like(active)
        for axis in range(active.ndim):
            near |= np.roll(active, 1, axis=axis)
            near |= np.roll(active, -1, axis=axis)
        states[(~active) & near] = STATE_TRANSITION
    return states


def sigma_field(states, block):
    """Per-mode weight sigma(k) (S1.1, Eq. S.1-S.3).

    ACTIVE blocks: 1.  FROZEN blocks: 0 (never used: they are not updated).
    TRANSITION blocks: product over the faces whose neighbouring block is
    FROZEN of w(distance of the mode from that face), i.e. w(i) for the
    lower face and w(B-1-i) for the upper face of each axis.
    """
    states = np.asarray(states)
    d = states.ndim
    nbs = states.shape
    dims = tuple(nb * b for nb, b in zip(nbs, block))
    sigma = np.zeros(dims, dtype=np.float64)
    w = [taper(b) for b in block]
    for bidx in np.ndindex(*nbs):
        st = states[bidx]
        sl = tuple(slice(i * b, (i + 1) * b) for i, b in zip(bidx, block))
        if st == STATE_ACTIVE:
            sigma[sl] = 1.0
        elif st == STATE_TRANSITION:
            local = np.ones(tuple(block), dtype=np.float64)
            for axis in range(d):
                shape = [1] * d
                shape[axis] = block[axis]
                lo = list(bidx)
                lo[axis] = (bidx[axis] - 1) % nbs[axis]
                hi = list(bidx)
                hi[axis] = (bidx[axis] + 1) % nbs[axis]
                if states[tuple(lo)] == STATE_FROZEN:
                    local = local * w[axis].reshape(shape)
                if states[tuple(hi)] == STATE_FROZEN:
                    local = local * w[axis][::-1].reshape(shape)
            sigma[sl] = local
    return sigma


def _state_field(states, block):
    """Expand per-block states to per-mode states."""
    out = np.asarray(states)
    for axis, b in enumerate(block):
        out = np.repeat(out, b, axis=axis)
    return out


# --------------------------------------------------------------------------------------
# Cahn-Hilliard semi-implicit Fourier step (conserved form, S3.1; semi-implicit, S4.2)
# --------------------------------------------------------------------------------------
def ch_real_field(c_hat):
    """c = Re(IFFT(c_hat))."""
    return np.real(ifftn(c_hat))


def ch_mass(c_hat):
    """Sum of c over the grid, in FP64."""
    return float(np.sum(ch_real_field(c_hat)))


def _ch_new(c_hat, k2, dt, kappa):
    c = ch_real_field(c_hat)
    g = c * c * c - c
    g_hat = fftn(g)
    return (c_hat - dt * k2 * g_hat) / (1.0 + dt * kappa * k2 * k2)


def ch_regular_step(c_hat, k2, dt, kappa):
    """Regular (dense) step: c_hat <- (c_hat - dt k^2 FFT(c^3 - c)) / (1 + dt kappa k^4)."""
    return _ch_new(c_hat, k2, dt, kappa)


def ch_masked_step(c_hat, states, block, k2, dt, kappa, sigma=None):
    """sp-DBA step: ACTIVE modes take the Regular result, TRANSITION modes
    c_hat + sigma (new - c_hat), FROZEN modes keep c_hat (S1.1, Eq. S.1)."""
    new = _ch_new(c_hat, k2, dt, kappa)
    if sigma is None:
        sigma = sigma_field(states, block)
    st = _state_field(states, block)
    out = np.where(st == STATE_ACTIVE, new, c_hat)
    tr = st == STATE_TRANSITION
    out[tr] = c_hat[tr] + sigma[tr] * (new[tr] - c_hat[tr])
    return out


class CHConfig:
    """Parameters of an adaptive Cahn-Hilliard run (all keyword-overridable)."""

    def __init__(self, dims, block, threshold=1e-6, reassess=10, dt=0.01, kappa=1.0,
                 mode=1, measure=MEASURE_MAXAMP, tau_rule=TAU_REL_MAX, transitions=True,
                 refresh_every=0, warmup_steps=0, force_dc=True, target_ratio=0.0, control_every=50,
                 control_eta=0.05):
        self.dims = tuple(int(x) for x in dims)
        self.block = tuple(int(x) for x in block)
        self.threshold = float(threshold)
        self.reassess = int(reassess)
        self.dt = float(dt)
        self.kappa = float(kappa)
        self.mode = int(mode)
        self.measure = int(measure)
        self.tau_rule = int(tau_rule)
        self.transitions = bool(transitions)
        self.refresh_every = int(refresh_every)
        self.warmup_steps = int(warmup_steps)
        self.force_dc = bool(force_dc)
        self.target_ratio = float(target_ratio)   # dynamic threshold control (S1.3), 0 = off
        self.control_every = int(control_every)
        self.control_eta = float(control_eta)


def assess_states(q, cfg, exclude_dc, threshold=None):
    """Measure, threshold and classify a transformed field; returns (states, tau, measure).
    `threshold` overrides cfg.threshold (the coefficient dynamic control adjusts)."""
    maxsq, sumsq = block_measures(q, cfg.block)
    measure = np.sqrt(maxsq if cfg.measure == MEASURE_MAXAMP else sumsq)
    tau = threshold_value(q, cfg.threshold if threshold is None else threshold, cfg.tau_rule, exclude_dc)
    states = classify(measure, tau, force_dc=cfg.force_dc, transitions=cfg.transitions)
    return states, tau, measure


def is_control_step(step, cfg):
    """Dynamic threshold control checks the ratio at every control_every-th step
    once the warm-up is over (S1.3; control starts after the full-activation
    stage, S3.2).  The step right after a check -- here the step at which the
    check is made, before its update -- runs with every block active."""
    return (getattr(cfg, "target_ratio", 0.0) > 0 and step > cfg.warmup_steps
            and step % cfg.control_every == 0)


def effective_states(assessed, step, cfg):
    """All blocks ACTIVE on warm-up, refresh and control steps (S1.3, S3.2), else the last assessment."""
    if step < cfg.warmup_steps or (cfg.refresh_every > 0 and step > 0
                                   and step % cfg.refresh_every == 0) or is_control_step(step, cfg):
        return np.full_like(assessed, STATE_ACTIVE)
    return assessed


def threshold_control(threshold, r, r_tar, eta):
    """One dynamic threshold-control decision (S1.3).

    r is the measured mean share of non-frozen (active + transition) blocks
    over the control interval and r_tar the target.  With q = r / r_tar:
    q > 2 doubles the threshold, q < 0.5 halves it; otherwise a deviation
    outside the relative deadband (q > 1 + eta or q < 1 - eta) scales it by
    1 + eta or 1 - eta; inside the deadband (edges included) it is kept.
    """
    q = r / r_tar
    if q > 2.0:
        return threshold * 2.0
    if q < 0.5:
        return threshold * 0.5
    if q > 1.0 + eta:
        return threshold * (1.0 + eta)
    if q < 1.0 - eta:
        return threshold * (1.0 - eta)
    return threshold


class ThresholdController:
    """The threshold coefficient of a run under dynamic control (S1.3).

    Each adaptive step (not a warm-up, refresh or control step) adds the
    number of non-frozen blocks of the states in force; at a control step the
    interval's mean share r = sum / (steps * nblocks) drives one
    threshold_control decision (when at least one adaptive step was seen) and
    the interval restarts.  `log` records (step, threshold) after each
    decision.
    """

    def __init__(self, cfg, nblocks):
        self.cfg = cfg
        self.nblocks = int(nblocks)
        self.threshold = float(cfg.threshold)
        self.sum_nonfrozen = 0
        self.steps = 0
        self.log = []

    def begin_step(self, step):
        """Called before the step's reassessment; returns the threshold in force."""
        if is_control_step(step, self.cfg) and self.steps > 0:
            r = float(self.sum_nonfrozen) / (float(self.steps) * float(self.nblocks))
            self.threshold = threshold_control(self.threshold, r, self.cfg.target_ratio, self.cfg.control_eta)
            self.sum_nonfrozen = 0
            self.steps = 0
            self.log.append((step, self.threshold))
        return self.threshold

    def end_step(self, step, states_in_force):
        """Called after the step with the assessed states in force (not the forced ones)."""
        forced = step < self.cfg.warmup_steps or (self.cfg.refresh_every > 0 and step > 0
                                                  and step % self.cfg.refresh_every == 0) \
            or is_control_step(step, self.cfg)
        if not forced:
            self.sum_nonfrozen += int(np.count_nonzero(np.asarray(states_in_force) != STATE_FROZEN))
            self.steps += 1


def run_ch(c0, cfg, steps, start_step=0, c_hat=None, on_assess=None, states=None, controller=None):
    """Advance a CH field `steps` steps.  Returns (c_hat, history) where history
    lists (step, states, tau) at each reassessment.  `on_assess(step, c_hat,
    states, tau)` may return replacement states (lock-step mask parity).  To
    continue a run, pass its c_hat, start_step, the states in force and its
    ThresholdController (one is made when cfg.target_ratio > 0)."""
    k2 = k_squared(cfg.dims)
    if c_hat is None:
        c_hat = fftn(np.asarray(c0, dtype=np.float64))
    if controller is None and getattr(cfg, "target_ratio", 0.0) > 0:
        controller = ThresholdController(cfg, np.prod(block_counts(cfg.dims, cfg.block)))
    history = []
    for n in range(start_step, start_step + steps):
        if cfg.mode == 0:
            c_hat = ch_regular_step(c_hat, k2, cfg.dt, cfg.kappa)
            continue
        thr = controller.begin_step(n) if controller is not None else None
        if states is None or n % cfg.reassess == 0:
            states, tau, _ = assess_states(c_hat, cfg, exclude_dc=True, threshold=thr)
            if on_assess is not None:
                repl = on_assess(n, c_hat, states, tau)
                if repl is not None:
                    states = repl
            history.append((n, states.copy(), tau))
        eff = effective_states(states, n, cfg)
        c_hat = ch_masked_step(c_hat, eff, cfg.block, k2, cfg.dt, cfg.kappa)
        if controller is not None:
            controller.end_step(n, states)
    return c_hat, history


# --------------------------------------------------------------------------------------
# Half-spectrum (real-to-complex) storage of a real CH field, block states on the
# stored half with conjugate neighbour activation (S1.2, Eq. S.4)
# --------------------------------------------------------------------------------------
def half_extent(n_last):
    """Stored x frequencies of a real field along its last axis: kx = 0 .. N/2 (N even)."""
    return n_last // 2 + 1


def rfftn_half(x):
    """The stored half of the DFT of a real field: X[..., kx] for kx = 0 .. N/2; the
    omitted half follows from X(-k) = conj X(k) (Eq. S.4)."""
    X = fftn(np.asarray(x, dtype=np.float64))
    return np.ascontiguousarray(X[..., : half_extent(X.shape[-1])])


def _negate_index(a, axes):
    """a[j] -> a[(-j) mod N] along each of `axes`."""
    for axis in axes:
        a = np.roll(np.flip(a, axis=axis), 1, axis=axis)
    return a


def hermitian_extend(h, dims):
    """Full spectrum of a half-stored one: kx = 0 .. N/2 as stored, kx = N/2+1 .. N-1 by
    Eq. S.4, X(k_other, kx) = conj X(-k_other, N - kx)."""
    dims = tuple(int(x) for x in dims)
    m = dims[-1] // 2
    full = np.zeros(dims, dtype=np.complex128)
    full[..., : m + 1] = h
    mirror = _negate_index(np.asarray(h)[..., 1:m][..., ::-1], range(len(dims) - 1))
    full[..., m + 1:] = np.conj(mirror)
    return full


def ch_real_field_half(h, dims):
    """c of a half-stored spectrum: Re(IFFT) of its Hermitian extension.  Where the stored
    kx = 0 and kx = N/2 planes are not conjugate-symmetric within themselves, Re(.) keeps
    their Hermitian part, as a complex-to-real transform does."""
    return np.real(ifftn(hermitian_extend(h, dims)))


def half_block_counts(dims, block):
    """Block grid of the stored half spectrum: the full grid's counts on every axis but
    the last; there the columns kx = 0 .. N/2 take N/(2B) + 1 blocks of B columns, the
    last holding the column kx = N/2 alone (its other B - 1 columns are absent)."""
    dims = tuple(int(x) for x in dims)
    block = tuple(int(x) for x in block)
    n, b = dims[-1], block[-1]
    if n % (2 * b) != 0:
        raise ValueError("the half map needs 2 B | N along the last axis (B=%d, N=%d)" % (b, n))
    return tuple(block_counts(dims[:-1], block[:-1])) + (n // (2 * b) + 1,)


def _pad_half(a, dims, block):
    """A half-grid array padded along its last axis to whole blocks with zeros."""
    nbs = half_block_counts(dims, block)
    out = np.zeros(a.shape[:-1] + (nbs[-1] * block[-1],), dtype=a.dtype)
    out[..., : a.shape[-1]] = a
    return out


def half_block_measures(h, dims, block):
    """Per-block max |q|^2 and sum |q|^2 (FP64) on the half map (absent modes count as 0)."""
    sq = _blockify(_pad_half(_mode_sq(h), dims, block), block)
    axes = tuple(range(1, sq.ndim, 2))
    return sq.max(axis=axes), sq.sum(axis=axes)


def half_neighbour(idx, axis, d, nbs):
    """Face neighbour (d = -1 / +1) along `axis` of block `idx` of a half map (S1.2).

    Every axis but the last wraps periodically.  Along the last axis a neighbour inside
    the stored half is taken directly; one in the omitted half -- left of kx = 0 or right
    of the Nyquist block -- is replaced by its conjugate counterpart (Eq. S.4): the block
    that holds most of the negated modes, i.e. the other axes' block indices mirrored
    (b -> nb - 1 - b) with block 0 on the last axis (across kx = 0, the symmetry
    boundary, whose partner block is then activated) or the block just below the Nyquist
    block (past kx = N/2, whose conjugates kx = N/2 - B .. N/2 - 1 fill that block)."""
    idx = list(idx)
    last = len(nbs) - 1
    if axis != last:
        idx[axis] = (idx[axis] + d) % nbs[axis]
        return tuple(idx)
    v = idx[last] + d
    if 0 <= v < nbs[last]:
        idx[last] = v
        return tuple(idx)
    for a in range(last):
        idx[a] = nbs[a] - 1 - idx[a]
    idx[last] = 0 if v < 0 else nbs[last] - 2
    return tuple(idx)


def classify_half(measure, tau, force_dc=False, transitions=True):
    """Block states of a half map: ACTIVE iff measure >= tau (the block holding k = 0
    forced ACTIVE when force_dc, S6.1).  With transitions every ACTIVE block requests
    activation of its face neighbours -- half_neighbour, so a neighbour in the omitted
    half is replaced by its conjugate counterpart (S1.2) -- and each requested block
    that is not ACTIVE becomes TRANSITION; the rest are FROZEN.  (Past the Nyquist
    block the relation is not symmetric: the block requested there does not request
    the Nyquist block back.)"""
    active = np.asarray(measure, dtype=np.float64) >= tau
    if force_dc:
        active.flat[0] = True
    states = np.where(active, STATE_ACTIVE, STATE_FROZEN).astype(np.uint8)
    if transitions:
        nbs = active.shape
        for idx in zip(*np.nonzero(active)):
            for axis in range(len(nbs)):
                for d in (-1, 1):
                    nb = half_neighbour(idx, axis, d, nbs)
                    if not active[nb]:
                        states[nb] = STATE_TRANSITION
    return states


def sigma_field_half(states, dims, block):
    """Per-mode sigma on the stored half grid (S1.1, Eq. S.1-S.3 with the half map's
    neighbours): 1 in ACTIVE blocks, 0 in FROZEN ones, and in TRANSITION blocks the
    product over faces whose neighbour (half_neighbour) is FROZEN of w(i) (lower face)
    or w(B-1-i) (upper face), i the mode's position in the block."""
    states = np.asarray(states)
    nbs = states.shape
    d = states.ndim
    w = [taper(b) for b in block]
    sigma = np.zeros(tuple(nb * b for nb, b in zip(nbs, block)), dtype=np.float64)
    for bidx in np.ndindex(*nbs):
        st = states[bidx]
        sl = tuple(slice(i * b, (i + 1) * b) for i, b in zip(bidx, block))
        if st == STATE_ACTIVE:
            sigma[sl] = 1.0
        elif st == STATE_TRANSITION:
            local = np.ones(tuple(block), dtype=np.float64)
            for axis in range(d):
                shape = [1] * d
                shape[axis] = block[axis]
                if states[half_neighbour(bidx, axis, -1, nbs)] == STATE_FROZEN:
                    local = local * w[axis].reshape(shape)
                if states[half_neighbour(bidx, axis, +1, nbs)] == STATE_FROZEN:
                    local = local * w[axis][::-1].reshape(shape)
            sigma[sl] = local
    return np.ascontiguousarray(sigma[..., : half_extent(dims[-1])])


def k_squared_half(dims, dx=1.0):
    """|k|^2 on the stored half grid (kx = 0 .. N/2)."""
    return np.ascontiguousarray(k_squared(dims, dx)[..., : half_extent(dims[-1])])


def _ch_new_half(h, dims, k2h, dt, kappa):
    c = ch_real_field_half(h, dims)
    g_hat = rfftn_half(c * c * c - c)
    return (h - dt * k2h * g_hat) / (1.0 + dt * kappa * k2h * k2h)


def ch_regular_step_half(h, dims, k2h, dt, kappa):
    """Regular step on the stored half (the same update as ch_regular_step, mode by mode)."""
    return _ch_new_half(h, dims, k2h, dt, kappa)


def ch_masked_step_half(h, states, dims, block, k2h, dt, kappa, sigma=None):
    """sp-DBA step on the stored half with half-map states (S1.1, Eq. S.1; S1.2)."""
    new = _ch_new_half(h, dims, k2h, dt, kappa)
    if sigma is None:
        sigma = sigma_field_half(states, dims, block)
    st = np.ascontiguousarray(_state_field(states, block)[..., : half_extent(dims[-1])])
    out = np.where(st == STATE_ACTIVE, new, h)
    tr = st == STATE_TRANSITION
    out[tr] = h[tr] + sigma[tr] * (new[tr] - h[tr])
    return out


def assess_states_half(h, cfg, exclude_dc, threshold=None):
    """Measure, threshold and classify a half-stored spectrum; returns (states, tau, measure)."""
    maxsq, sumsq = half_block_measures(h, cfg.dims, cfg.block)
    measure = np.sqrt(maxsq if cfg.measure == MEASURE_MAXAMP else sumsq)
    tau = threshold_value(h, cfg.threshold if threshold is None else threshold, cfg.tau_rule, exclude_dc)
    states = classify_half(measure, tau, force_dc=cfg.force_dc, transitions=cfg.transitions)
    return states, tau, measure


def run_ch_half(c0, cfg, steps, start_step=0, h=None, on_assess=None, states=None, controller=None):
    """run_ch with the spectrum stored as its half (kx = 0 .. N/2) and block states on the
    half map; returns (h, history).  Same schedule (reassessment, refresh, warm-up,
    dynamic control) and callbacks as run_ch."""
    dims = cfg.dims
    k2h = k_squared_half(dims)
    if h is None:
        h = rfftn_half(c0)
    if controller is None and getattr(cfg, "target_ratio", 0.0) > 0:
        controller = ThresholdController(cfg, np.prod(half_block_counts(dims, cfg.block)))
    history = []
    for n in range(start_step, start_step + steps):
        if cfg.mode == 0:
            h = ch_regular_step_half(h, dims, k2h, cfg.dt, cfg.kappa)
            continue
        thr = controller.begin_step(n) if controller is not None else None
        if states is None or n % cfg.reassess == 0:
            states, tau, _ = assess_states_half(h, cfg, exclude_dc=True, threshold=thr)
            if on_assess is not None:
                repl = on_assess(n, h, states, tau)
                if repl is not None:
                    states = repl
            history.append((n, states.copy(), tau))
        eff = effective_states(states, n, cfg)
        h = ch_masked_step_half(h, eff, dims, cfg.block, k2h, cfg.dt, cfg.kappa)
        if controller is not None:
            controller.end_step(n, states)
    return h, history


# --------------------------------------------------------------------------------------
# Scalar NLS split-step Fourier (S5.1-S5.2 with M = 1, alpha = 0)
# --------------------------------------------------------------------------------------
def nls_omega(n, dt_sample):
    """Angular frequency of each FFT bin: 2 pi j / (n dt) with j in FFT order."""
    return wavenumbers(n, dt_sample)


def nls_half_factor(omega, beta2, h):
    """Linear half-step propagator exp((i beta2 omega^2 / 2) h / 2) for E(t) = (1/N) sum E~ e^{+i w t}
    (S5.2, alpha = 0, no mode coupling)."""
    return np.exp(1j * beta2 * omega * omega * h / 4.0)


def nls_kerr(E, gamma, h):
    """Time-domain Kerr step E exp(i gamma |E|^2 h) (scalar field: no Manakov 8/9)."""
    p = np.real(E) ** 2 + np.imag(E) ** 2
    return E * np.exp(1j * gamma * p * h)


def nls_masked_half(Et, states, block, H, sigma=None):
    """Blockwise linear half-step: ACTIVE E~ H, TRANSITION E~ + sigma (E~ H - E~), FROZEN E~."""
    new = Et * H
    if states is None:
        return new
    if sigma is None:
        sigma = sigma_field(states, block)
    st = _state_field(states, block)
    out = np.where(st == STATE_ACTIVE, new, Et)
    tr = st == STATE_TRANSITION
    out[tr] = Et[tr] + sigma[tr] * (new[tr] - Et[tr])
    return out


def nls_regular_step(E, H, gamma, h):
    """One symmetric split step, literal order: L/2 -> N -> L/2 with 4 transforms."""
    return nls_masked_step(E, None, None, H, gamma, h)


def nls_masked_step(E, states, block, H, gamma, h, sigma=None):
    Et = fftn(E)
    Et = nls_masked_half(Et, states, block, H, sigma)
    E = ifftn(Et)
    E = nls_kerr(E, gamma, h)
    Et = fftn(E)
    Et = nls_masked_half(Et, states, block, H, sigma)
    return ifftn(Et)


class NLSConfig:
    def __init__(self, n, block, threshold=1e-6, reassess=10, beta2=-21.7, gamma=1.3, h=0.1,
                 dt_sample=1.0, mode=1, measure=MEASURE_MAXAMP, tau_rule=TAU_REL_MAX,
                 transitions=True, refresh_every=0, warmup_steps=0, target_ratio=0.0, control_every=50,
                 control_eta=0.05):
        self.dims = (int(n),)
        self.block = (int(block),)
        self.threshold = float(threshold)
        self.reassess = int(reassess)
        self.beta2 = float(beta2)
        self.gamma = float(gamma)
        self.h = float(h)
        self.dt_sample = float(dt_sample)
        self.mode = int(mode)
        self.measure = int(measure)
        self.tau_rule = int(tau_rule)
        self.transitions = bool(transitions)
        self.refresh_every = int(refresh_every)
        self.warmup_steps = int(warmup_steps)
        self.force_dc = False
        self.target_ratio = float(target_ratio)   # dynamic threshold control (S1.3), 0 = off
        self.control_every = int(control_every)
        self.control_eta = float(control_eta)


def run_nls(E0, cfg, steps, on_assess=None, controller=None):
    """Propagate E0 by `steps` split steps; states are assessed on FFT(E) at the
    start of a step, every `reassess` steps (S5.3: total spectral power, M = 1).
    With cfg.target_ratio > 0 the threshold follows dynamic control (S1.3)."""
    n = cfg.dims[0]
    H = nls_half_factor(nls_omega(n, cfg.dt_sample), cfg.beta2, cfg.h)
    E = np.asarray(E0, dtype=np.complex128)
    if controller is None and cfg.target_ratio > 0:
        controller = ThresholdController(cfg, n // cfg.block[0])
    history = []
    states = None
    for s in range(steps):
        if cfg.mode == 0:
            E = nls_regular_step(E, H, cfg.gamma, cfg.h)
            continue
        thr = controller.begin_step(s) if controller is not None else None
        if states is None or s % cfg.reassess == 0:
            states, tau, _ = assess_states(fftn(E), cfg, exclude_dc=False, threshold=thr)
            if on_assess is not None:
                repl = on_assess(s, E, states, tau)
                if repl is not None:
                    states = repl
            history.append((s, states.copy(), tau))
        eff = effective_states(states, s, cfg)
        E = nls_masked_step(E, eff, cfg.block, H, cfg.gamma, cfg.h)
        if controller is not None:
            controller.end_step(s, states)
    return E, history


# --------------------------------------------------------------------------------------
# Reaction-cross-diffusion with M components (S4.1-S4.3)
# --------------------------------------------------------------------------------------
def rcd_diffusion_matrix(M, d_diag, d_cross):
    """Symmetric circulant cross-diffusion matrix (S4.1): D_ii = d_diag + 2 d_cross,
    D_{i,i+1} = D_{i,i-1} = -d_cross with periodic component index; for M = 2
    the two neighbours coincide and the single off-diagonal entry is -d_cross."""
    D = np.zeros((M, M), dtype=np.float64)
    for i in range(M):
        D[i, i] = d_diag + 2.0 * d_cross
        if M > 1:
            D[i, (i + 1) % M] = -d_cross
            D[i, (i - 1) % M] = -d_cross
    return D


def rcd_interaction_matrix(M, alpha, beta):
    """Off-diagonal Lotka-Volterra interactions alpha_ij (S4.1): beta + alpha for the
    two neighbouring components (periodic index; one entry for M = 2), beta for
    every other j != i; zero diagonal (self-limitation is a_i)."""
    A = np.full((M, M), float(beta), dtype=np.float64)
    np.fill_diagonal(A, 0.0)
    for i in range(M):
        if M > 1:
            A[i, (i + 1) % M] = beta + alpha
            A[i, (i - 1) % M] = beta + alpha
    return A


def rcd_reaction(u, r, a, A):
    """Generalised Lotka-Volterra reaction R_i(u) = u_i (r_i - a_i u_i - sum_{j != i}
    alpha_ij u_j) (S4.1), u of shape (M, ...) (component first)."""
    M = u.shape[0]
    inter = np.tensordot(A, u, axes=(1, 0))          # sum_j alpha_ij u_j (alpha_ii = 0)
    r = np.asarray(r, dtype=np.float64).reshape((M,) + (1,) * (u.ndim - 1))
    a = np.asarray(a, dtype=np.float64).reshape((M,) + (1,) * (u.ndim - 1))
    return u * (r - a * u - inter)


def rcd_homogeneous_state(M, r, a, alpha, beta):
    """The equal-concentration fixed point of the reaction: r = u (a + sum_{j != i} alpha_ij)."""
    return float(r) / (float(a) + float(rcd_interaction_matrix(M, alpha, beta)[0].sum()))


def rcd_eigen(D):
    """D = V diag(lam) V^T (symmetric D; V orthogonal), computed once (S4.3)."""
    lam, V = np.linalg.eigh(D)
    return lam, V


def rcd_update_direct(b, k2, dt, D):
    """u_new(k) = (I + dt k^2 D)^{-1} b(k) for every mode (S4.2), one dense M x M
    solve per distinct |k|^2; b of shape (M, ...) complex."""
    M = b.shape[0]
    flat_b = b.reshape(M, -1)
    flat_k2 = np.asarray(k2, dtype=np.float64).reshape(-1)
    out = np.empty_like(flat_b)
    for val in np.unique(flat_k2):
        sel = flat_k2 == val
        A = np.eye(M) + dt * val * D
        out[:, sel] = np.linalg.solve(A, flat_b[:, sel])
    return out.reshape(b.shape)


def rcd_update_eigen(b, k2, dt, V, lam):
    """The same update through the eigendecomposition (S4.3):
    V (I + dt k^2 Lambda)^{-1} V^T b."""
    M = b.shape[0]
    y = np.tensordot(V.T, b, axes=(1, 0))
    den = 1.0 + dt * np.asarray(k2, dtype=np.float64)[None, ...] * lam.reshape((M,) + (1,) * (b.ndim - 1))
    return np.tensordot(V, y / den, axes=(1, 0))


def rcd_mode_amplitude_sq(q):
    """A(k)^2 = (1/M) sum_m |q_m(k)|^2 (S4.2: component RMS Fourier amplitude), FP64."""
    return np.sum(_mode_sq(q), axis=0) / float(q.shape[0])


class RCDConfig:
    """Parameters of an RCD run (S4.2 defaults: dx = 0.5, dt = 0.01, D_diag = 0.5,
    D_cross = 0.05, alpha = 1, beta = 0.3, r_i = a_i = 1)."""

    def __init__(self, dims, block, M, threshold=1e-6, reassess=10, dt=0.01, dx=0.5, d_diag=0.5,
                 d_cross=0.05, alpha=1.0, beta=0.3, r=1.0, a=1.0, mode=1, tau_rule=TAU_REL_MAX,
                 transitions=True, refresh_every=0, warmup_steps=0, force_dc=True, eigen=True,
                 target_ratio=0.0, control_every=50, control_eta=0.1):
        self.dims = tuple(int(x) for x in dims)
        self.block = tuple(int(x) for x in block)
        self.M = int(M)
        self.threshold = float(threshold)
        self.reassess = int(reassess)
        self.dt, self.dx = float(dt), float(dx)
        self.d_diag, self.d_cross = float(d_diag), float(d_cross)
        self.alpha, self.beta, self.r, self.a = float(alpha), float(beta), float(r), float(a)
        self.mode = int(mode)
        self.measure = MEASURE_MAXAMP
        self.tau_rule = int(tau_rule)
        self.transitions = bool(transitions)
        self.refresh_every = int(refresh_every)
        self.warmup_steps = int(warmup_steps)
        self.force_dc = bool(force_dc)
        self.eigen = bool(eigen)
        self.target_ratio = float(target_ratio)
        self.control_every = int(control_every)
        self.control_eta = float(control_eta)


def rcd_assess_states(u_hat, cfg, threshold=None):
    """States from the component RMS amplitude (S4.2): a block is ACTIVE when one of
    its modes has A(k) >= tau; the state applies to all M components.  tau is
    threshold * max_{k != 0} A(k) (REL_MAX) or threshold (ABS)."""
    a2 = rcd_mode_amplitude_sq(u_hat)
    blk = _blockify(a2, cfg.block)
    maxsq = blk.max(axis=tuple(range(1, blk.ndim, 2)))
    measure = np.sqrt(maxsq)
    thr = cfg.threshold if threshold is None else threshold
    if cfg.tau_rule == TAU_ABS:
        tau = float(thr)
    else:
        a2x = a2.copy()
        a2x.flat[0] = 0.0
        tau = float(thr) * math.sqrt(float(a2x.max()))
    states = classify(measure, tau, force_dc=cfg.force_dc, transitions=cfg.transitions)
    return states, tau, measure


def rcd_real_field(u_hat):
    """u_m = Re(IFFT(u_hat_m)) for every component."""
    return np.stack([np.real(ifftn(q)) for q in u_hat])


def rcd_new(u_hat, cfg, k2, D, eig):
    """The update core of every mode: (I + dt k^2 D)^{-1} [u_hat + dt FFT(R(u))] (S4.2)."""
    u = rcd_real_field(u_hat)
    A = rcd_interaction_matrix(cfg.M, cfg.alpha, cfg.beta)
    R = rcd_reaction(u, np.full(cfg.M, cfg.r), np.full(cfg.M, cfg.a), A)
    b = u_hat + cfg.dt * np.stack([fftn(x) for x in R])
    if cfg.eigen:
        return rcd_update_eigen(b, k2, cfg.dt, eig[1], eig[0])
    return rcd_update_direct(b, k2, cfg.dt, D)


def rcd_masked_step(u_hat, states, cfg, k2, D, eig, sigma=None):
    """sp-DBA step: ACTIVE blocks take the update core's result for all M
    components, TRANSITION blocks u + sigma (new - u), FROZEN blocks keep u (S4.2)."""
    new = rcd_new(u_hat, cfg, k2, D, eig)
    if states is None:
        return new
    if sigma is None:
        sigma = sigma_field(states, cfg.block)
    st = _state_field(states, cfg.block)
    out = np.where(st[None] == STATE_ACTIVE, new, u_hat)
    tr = st == STATE_TRANSITION
    out[:, tr] = u_hat[:, tr] + sigma[tr][None, :] * (new[:, tr] - u_hat[:, tr])
    return out


def run_rcd(u0, cfg, steps, u_hat=None, on_assess=None, controller=None):
    """Advance M real component fields u0 (M, *dims) `steps` steps; returns (u_hat,
    history of (step, states, tau)).  Same state schedule as run_ch."""
    k2 = k_squared(cfg.dims, cfg.dx)
    D = rcd_diffusion_matrix(cfg.M, cfg.d_diag, cfg.d_cross)
    eig = rcd_eigen(D)
    if u_hat is None:
        u_hat = np.stack([fftn(np.asarray(x, dtype=np.float64)) for x in u0])
    if controller is None and cfg.target_ratio > 0:
        controller = ThresholdController(cfg, np.prod(block_counts(cfg.dims, cfg.block)))
    history = []
    states = None
    for n in range(steps):
        if cfg.mode == 0:
            u_hat = rcd_masked_step(u_hat, None, cfg, k2, D, eig)
            continue
        thr = controller.begin_step(n) if controller is not None else None
        if states is None or n % cfg.reassess == 0:
            states, tau, _ = rcd_assess_states(u_hat, cfg, threshold=thr)
            if on_assess is not None:
                repl = on_assess(n, u_hat, states, tau)
                if repl is not None:
                    states = repl
            history.append((n, states.copy(), tau))
        eff = effective_states(states, n, cfg)
        u_hat = rcd_masked_step(u_hat, eff, cfg, k2, D, eig)
        if controller is not None:
            controller.end_step(n, states)
    return u_hat, history


# --------------------------------------------------------------------------------------
# Metrics (S5.3)
# --------------------------------------------------------------------------------------
def rel_l2(x, ref):
    """||x - ref||_2 / ||ref||_2 in FP64."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    num = np.sqrt(np.sum(np.abs(x.astype(np.complex128) - ref.astype(np.complex128)) ** 2))
    den = np.sqrt(np.sum(np.abs(ref.astype(np.complex128)) ** 2))
    return float(num / den)


def nmse_db(E, E_tx):
    """NMSE(dB) = 10 log10( sum |E - E_tx|^2 / sum |E_tx|^2 )."""
    E = np.asarray(E, dtype=np.complex128)
    E_tx = np.asarray(E_tx, dtype=np.complex128)
    return float(10.0 * np.log10(np.sum(np.abs(E - E_tx) ** 2) / np.sum(np.abs(E_tx) ** 2)))


def field_corr(E, E_tx):
    """|sum E^H E_tx| / (||E|| ||E_tx||)."""
    E = np.asarray(E, dtype=np.complex128)
    E_tx = np.asarray(E_tx, dtype=np.complex128)
    num = abs(np.sum(np.conj(E) * E_tx))
    return float(num / math.sqrt(np.sum(np.abs(E) ** 2) * np.sum(np.abs(E_tx) ** 2)))
