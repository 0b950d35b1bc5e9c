"""Constants of the method, with the passage each one comes from (oracle copy).

Test infrastructure only.  The CUDA path receives the same numbers through its own config
struct; nothing here is shared with it.
"""
from dataclasses import dataclass, field

import numpy as np

# Table 2 (App. A.3): reward weights, each multiplied by dt.
W_LIN_VEL = 1.0        # phi(v*_xy - v_xy)
W_ANG_VEL = 0.5        # phi(w*_z - w_z)
W_VZ = 4.0             # -v_z^2
W_WXY = 0.05           # -|w_xy|^2
W_JOINT = 0.001        # -|qdd|^2 - |qd|^2
W_TORQUE = 0.00002     # -|tau|^2
W_ACTION_RATE = 0.25   # -|a_t - a_{t-1}|^2
W_COLLISION = 0.001    # -n_collision
W_AIR_TIME = 2.0       # sum_f (t_air,f - 0.5) on first contact
PHI_SCALE = 0.25       # phi(x) = exp(-|x|^2 / 0.25)
AIR_TIME_TARGET = 0.5

# Table 4 (App. A.5): uniform observation-noise half-widths.
NOISE_LIN_VEL = 0.01
NOISE_ANG_VEL = 0.2
NOISE_GRAVITY = 0.05
NOISE_CMD = 0.0
NOISE_DOF_POS = 0.01
NOISE_DOF_VEL = 1.5
NOISE_ACTIONS = 0.0    # previous actions are not listed in Table 4
NOISE_HEIGHT = 0.1

# Table 3 (App. A.4) and Algorithm 1.
GAMMA = 0.99
LAM = 0.95
CLIP = 0.2
ENTROPY_COEF = 0.01
KL_TARGET = 0.01
EPOCHS = 5
MINIBATCHES = 4
LR_INIT = 1e-3
LR_MIN = 1e-5
LR_MAX = 1e-2
LR_FACTOR = 1.5
VALUE_COEF = 1.0
ADAM_BETA1 = 0.9
ADAM_BETA2 = 0.999
ADAM_EPS = 1e-8
ADV_EPS = 1e-8

# Slots of the per-(env, step) random key (counter-based generator, see oracle.rng).
SLOTS_PER_SUBSTEP = 32       # substep k uses slots 32k + {0..11 qd, 12..14 v, 15..17 w, 18..19 g, 20 z}
SLOT_CRASH = 128
SLOT_COLLISIONS = 129
SLOT_LOOPBACK = 130
SLOT_PUSH_X = 131
SLOT_PUSH_Y = 132
SLOT_CMD = 133               # 133, 134, 135
SLOT_HEADING = 136           # 136, 137
SLOT_EPLEN = 138
SLOT_OBS_NOISE = 256         # obs column k uses word 256 + k // 2 (hi half for even k, lo for odd)

# Foot contact schedule of the stand-in (integer): period 40 policy steps, half duty.
CONTACT_PERIOD = 40
CONTACT_DUTY = 20
CONTACT_PHASE = (0, 20, 20, 0)
CONTACT_ENV_STRIDE = 7


@dataclass
class EnvConfig:
    num_envs: int = 64
    act_dim: int = 12
    kp: float = 80.0               # PD gains of the measured workload (Sec. 3.2 PD controller)
    kd: float = 2.0
    action_scale: float = 0.5      # q* = q_def + action_scale * a (Sec. 3.2: actions are joint targets)
    dt: float = 0.02               # 50 Hz policy (App. A.1.1)
    sim_dt: float = 0.005          # 4 simulation steps per policy step (App. A.1.1)
    decimation: int = 4
    max_episode_len: int = 1000    # 20 s time-out (Sec. 2.2.1)
    num_levels: int = 10           # curriculum rows (Sec. 3.1)
    num_cols: int = 20             # terrain-type columns
    tile_size: float = 8.0         # 8 m tiles (Sec. 3.1)
    hf_res: float = 0.1            # heightfield resolution
    grid_x: int = 17               # height-sample grid (Sec. 3.2 measures the terrain on a grid)
    grid_y: int = 11
    grid_spacing: float = 0.1
    gamma: float = GAMMA           # for the time-out bootstrap (Sec. 2.2.2)
    noise_on: bool = True          # Table 4
    push_on: bool = True           # Sec. 3.3: pushes every 10 s, up to +-1 m/s in x and y
    push_interval: int = 500
    push_vel: float = 1.0
    cmd_range: tuple = (1.0, 1.0, 1.0)
    crash_threshold: int = 9170000  # stand-in: P(crash) per step = threshold / 2^32
    seed: int = 0
    q_def: np.ndarray = field(default_factory=lambda: np.zeros(12, np.float32))

    @property
    def num_heights(self):
        return self.grid_x * self.grid_y

    @property
    def obs_dim(self):
        return 48 + self.num_heights

    @property
    def cells_per_tile(self):
        return int(round(self.tile_size / self.hf_res))

    @property
    def hf_shape(self):
        c = self.cells_per_tile
        return (self.num_levels * c, self.num_cols * c)

    def noise_scales(self):
        """Per-column noise half-width of the observation vector (Table 4)."""
        s = np.zeros(self.obs_dim)
        s[0:3] = NOISE_LIN_VEL
        s[3:6] = NOISE_ANG_VEL
        s[6:9] = NOISE_GRAVITY
        s[9:12] = NOISE_CMD
        s[12:24] = NOISE_DOF_POS
        s[24:36] = NOISE_DOF_VEL
        s[36:48] = NOISE_ACTIONS
        s[48:] = NOISE_HEIGHT
        return s


@dataclass
class PPOConfig:
    gamma: float = GAMMA
    lam: float = LAM
    clip: float = CLIP
    entropy_coef: float = ENTROPY_COEF
    value_coef: float = VALUE_COEF
    kl_target: float = KL_TARGET
    lr_init: float = LR_INIT
    lr_min: float = LR_MIN
    lr_max: float = LR_MAX
    epochs: int = EPOCHS
    minibatches: int = MINIBATCHES
    seed: int = 0
