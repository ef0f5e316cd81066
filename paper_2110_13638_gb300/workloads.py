"""Seeded synthetic workloads: network graphs, FP64 weights and slot data.

This module holds no CKKS arithmetic.  It produces the plain inputs that both
the CUDA path and the CPU oracle consume (numpy PCG64 generators):

  cfg0  dense 8->4 then x^2, 8 ciphertexts x 4096 samples, U[-1,1] data,
        weights N(0, 0.5) (std 0.5), weight seed 0, data seed 100
  cfg1  CNN on 28x28x1 images, U[0,1] pixels, 784 ciphertexts x 8192 samples:
        conv 5 filters 5x5 stride 2 (720 outputs) -> sigmoid fit -> dense
        720->100 -> sigmoid fit -> dense 100->10; He-normal weights, seed 1,
        data seed 101 (stands in for Fashion-MNIST, Sec. 3.2)
  cfg2  yield MLP, 64 features (52 lognormal(0,1) lagged yields + 12 N(0,1)
        weather covariates) x 8192 samples: dense 64->128 -> sigmoid fit ->
        128->32 -> sigmoid fit -> 32->1; Xavier-normal weights, seed 2, data
        seed 102 (stands in for the proprietary strawberry data, Sec. 3.3)

Biases are zero in the three networks (the paper does not give them); the
`mini_*` builders make small graphs with nonzero biases for parity tests.

Graph format (plain dict):
  nodes: list of {"kind": "input"|"linear"|"poly"|"square"|"add"|"output", ...}
         linear: n_out, row_ptr (uint32), col_idx (uint32), weight (float64),
                 bias (float64[n_out]); poly: coeffs [a0, a1, a2, a3]
  edges: list of (src, dst) in edge order
"""
import numpy as np


def sigmoid_fit(lo=-5.0, hi=5.0, npts=1001):
    """Degree-3 least-squares fit of 1/(1+e^-x) on npts equispaced points
    (the form of Eq. sigmoid_approximate)."""
    x = np.linspace(lo, hi, npts)
    y = 1.0 / (1.0 + np.exp(-x))
    A = np.stack([np.ones_like(x), x, x * x, x * x * x], axis=1)
    c, *_ = np.linalg.lstsq(A, y, rcond=None)
    return [float(v) for v in c]


def dense_csr(W):
    """Dense weight matrix [n_out][n_in] -> CSR arrays."""
    n_out, n_in = W.shape
    row_ptr = np.arange(0, n_out * n_in + 1, n_in, dtype=np.uint32)
    col_idx = np.tile(np.arange(n_in, dtype=np.uint32), n_out)
    return row_ptr, col_idx, np.ascontiguousarray(W.reshape(-1), dtype=np.float64)


def conv_csr(K, H, W_, stride):
    """Valid cross-correlation of one HxW_ channel with filters K[f][kh][kw]
    as a sparse linear map; output index = f*(OH*OW) + r*OW + c, input index
    = row*W_ + col."""
    F, kh, kw = K.shape
    OH = (H - kh) // stride + 1
    OW = (W_ - kw) // stride + 1
    rows, cols, vals = [0], [], []
    for f in range(F):
        for r in range(OH):
            for c in range(OW):
                for dr in range(kh):
                    for dc in range(kw):
                        cols.append((r * stride + dr) * W_ + (c * stride + dc))
                        vals.append(K[f, dr, dc])
                rows.append(len(cols))
    return (np.array(rows, dtype=np.uint32), np.array(cols, dtype=np.uint32),
            np.array(vals, dtype=np.float64), F * OH * OW)


def _linear(row_ptr, col_idx, weight, bias):
    return {"kind": "linear", "n_out": len(row_ptr) - 1, "row_ptr": row_ptr,
            "col_idx": col_idx, "weight": weight,
            "bias": np.ascontiguousarray(bias, dtype=np.float64)}


def chain_graph(n_in, blocks):
    nodes = [{"kind": "input", "n": n_in}] + blocks + [{"kind": "output"}]
    edges = [(i, i + 1) for i in range(len(nodes) - 1)]
    return {"nodes": nodes, "edges": edges}


def cfg0(n_slots=4096, weight_seed=0, data_seed=100, n_in=8, n_out=4):
    rng = np.random.Generator(np.random.PCG64(weight_seed))
    W = rng.normal(0.0, 0.5, size=(n_out, n_in))
    g = chain_graph(n_in, [_linear(*dense_csr(W), np.zeros(n_out)), {"kind": "square"}])
    drng = np.random.Generator(np.random.PCG64(data_seed))
    x = drng.uniform(-1.0, 1.0, size=(n_in, n_slots))
    return g, x


def cfg1(n_slots=8192, weight_seed=1, data_seed=101, side=28, filters=5, k=5,
         stride=2, hidden=100, classes=10):
    rng = np.random.Generator(np.random.PCG64(weight_seed))
    K = rng.normal(0.0, np.sqrt(2.0 / (k * k)), size=(filters, k, k))
    rp, ci, cv, n_conv = conv_csr(K, side, side, stride)
    W1 = rng.normal(0.0, np.sqrt(2.0 / n_conv), size=(hidden, n_conv))
    W2 = rng.normal(0.0, np.sqrt(2.0 / hidden), size=(classes, hidden))
    sig = sigmoid_fit()
    g = chain_graph(side * side, [
        _linear(rp, ci, cv, np.zeros(n_conv)),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W1), np.zeros(hidden)),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W2), np.zeros(classes)),
    ])
    drng = np.random.Generator(np.random.PCG64(data_seed))
    x = drng.uniform(0.0, 1.0, size=(side * side, n_slots))
    return g, x


def cfg2(n_slots=8192, weight_seed=2, data_seed=102, n_lag=52, n_weather=12,
         h1=128, h2=32, n_out=1):
    n_in = n_lag + n_weather
    rng = np.random.Generator(np.random.PCG64(weight_seed))
    W0 = rng.normal(0.0, np.sqrt(2.0 / (n_in + h1)), size=(h1, n_in))
    W1 = rng.normal(0.0, np.sqrt(2.0 / (h1 + h2)), size=(h2, h1))
    W2 = rng.normal(0.0, np.sqrt(2.0 / (h2 + n_out)), size=(n_out, h2))
    sig = sigmoid_fit()
    g = chain_graph(n_in, [
        _linear(*dense_csr(W0), np.zeros(h1)),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W1), np.zeros(h2)),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W2), np.zeros(n_out)),
    ])
    drng = np.random.Generator(np.random.PCG64(data_seed))
    lag = drng.lognormal(0.0, 1.0, size=(n_lag, n_slots))
    weather = drng.normal(0.0, 1.0, size=(n_weather, n_slots))
    return g, np.concatenate([lag, weather], axis=0)


def mini_cnn(n_slots, seed=7, side=8, filters=2, k=3, stride=2, hidden=5, classes=3):
    """A small cfg1-shaped network with nonzero biases, for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = rng.normal(0.0, np.sqrt(2.0 / (k * k)), size=(filters, k, k))
    rp, ci, cv, n_conv = conv_csr(K, side, side, stride)
    W1 = rng.normal(0.0, np.sqrt(2.0 / n_conv), size=(hidden, n_conv))
    W2 = rng.normal(0.0, np.sqrt(2.0 / hidden), size=(classes, hidden))
    b0 = rng.normal(0.0, 0.1, size=n_conv)
    b1 = rng.normal(0.0, 0.1, size=hidden)
    b2 = rng.normal(0.0, 0.1, size=classes)
    sig = sigmoid_fit()
    g = chain_graph(side * side, [
        _linear(rp, ci, cv, b0),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W1), b1),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W2), b2),
    ])
    x = rng.uniform(0.0, 1.0, size=(side * side, n_slots))
    return g, x


def cnn_relu(n_slots=8192, relu_q=4.0, **kw):
    """The CNN with the paper's ReLU approximation (Eq. relu_approximate,
    range q) as the activation after the convolution (Sec. 3.2 pairs the
    cross-correlation with ReLU) and the sigmoid fit after the dense layer."""
    g, x = cfg1(n_slots=n_slots, **kw)
    g["nodes"][2] = {"kind": "relu", "q": float(relu_q)}
    return g, x


def mini_cnn_relu(n_slots, seed=17, relu_q=3.0):
    """Small network with the three polynomial degrees: conv -> ReLU
    approximation (degree 2) -> dense -> linear sigmoid 0.5 + 0.197 x
    (degree 1, the linear part of Eq. sigmoid_approximate) -> dense."""
    g, x = mini_cnn(n_slots, seed=seed)
    g["nodes"][2] = {"kind": "relu", "q": float(relu_q)}
    g["nodes"][4] = {"kind": "poly", "coeffs": [0.5, 0.197]}
    return g, x


def with_rotation(g, after):
    """The chain graph g with a rotation (client refresh) node inserted after
    node `after`: the ciphertexts go back to the client, are decrypted and
    re-encrypted, and the rest of the network is a new parameter group."""
    nodes = g["nodes"][:after + 1] + [{"kind": "rotate"}] + g["nodes"][after + 1:]
    edges = [(i, i + 1) for i in range(len(nodes) - 1)]
    return {"nodes": nodes, "edges": edges}


def two_rings(n_slots=4096, seed=23, n_in=4, hidden=4, n_out=2):
    """dense -> square | rotation | dense -> sigmoid fit -> dense: groups of
    cost 2 (N = 8192) and 4 (N = 16384); the refresh widens the slots."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W0 = rng.normal(0.0, 0.5, size=(hidden, n_in))
    W1 = rng.normal(0.0, 0.5, size=(hidden, hidden))
    W2 = rng.normal(0.0, 0.5, size=(n_out, hidden))
    g = chain_graph(n_in, [_linear(*dense_csr(W0), np.zeros(hidden)), {"kind": "square"},
                           _linear(*dense_csr(W1), rng.normal(0.0, 0.1, size=hidden)),
                           {"kind": "poly", "coeffs": sigmoid_fit()},
                           _linear(*dense_csr(W2), np.zeros(n_out))])
    x = rng.uniform(-1.0, 1.0, size=(n_in, n_slots))
    return with_rotation(g, 2), x


def cnn_rotate(n_slots=8192, **kw):
    """The CNN with one rotation after the first sigmoid fit: groups of cost
    3 (conv, sigmoid) and 4 (dense, sigmoid, dense) instead of one of cost 7."""
    g, x = cfg1(n_slots=n_slots, **kw)
    return with_rotation(g, 2), x


def mini_cnn_rotate(n_slots, seed=7):
    g, x = mini_cnn(n_slots, seed=seed)
    return with_rotation(g, 2), x


def cnn_masquerade(n_ct, slots, seed=7, side=8, filters=2, k=3, stride=2, hidden=5, classes=3):
    """Kernel masquerading (Sec. 3.2): images packed side by side in each
    ciphertext (slot stride side^2), the convolution evaluated on the packed
    ciphertexts (rotations line every pixel up with its output slot, the
    merged mask-and-kernel vectors multiply slot-wise), a sigmoid fit on the
    packed result, then a rotation (client refresh) where the client re-packs
    the conv outputs one feature per ciphertext, images in slots, for the
    dense layers.  Parameter groups of cost 3 and 4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S = side * side
    images = slots // S
    K = rng.normal(0.0, np.sqrt(2.0 / (k * k)), size=(filters, k, k))
    OH = (side - k) // stride + 1
    n_feat = filters * OH * OH
    W1 = rng.normal(0.0, np.sqrt(2.0 / n_feat), size=(hidden, n_feat))
    W2 = rng.normal(0.0, np.sqrt(2.0 / hidden), size=(classes, hidden))
    b0 = rng.normal(0.0, 0.1, size=filters)
    geo = {"H": side, "W": side, "k": k, "stride": stride, "filters": filters, "images": images, "slot_stride": S}
    conv = dict(geo, kind="conv_packed", weight=K, bias=b0)
    sig = sigmoid_fit()
    nodes = [{"kind": "input", "n": n_ct}, conv, {"kind": "poly", "coeffs": sig},
             {"kind": "rotate", "relayout": geo},
             _linear(*dense_csr(W1), rng.normal(0.0, 0.1, size=hidden)),
             {"kind": "poly", "coeffs": sig},
             _linear(*dense_csr(W2), np.zeros(classes)), {"kind": "output"}]
    edges = [(i, i + 1) for i in range(len(nodes) - 1)]
    imgs = rng.uniform(0.0, 1.0, size=(n_ct * images, S))
    x = np.zeros((n_ct, slots))
    for i in range(n_ct):
        for b in range(images):
            x[i, b * S:(b + 1) * S] = imgs[i * images + b]
    return {"nodes": nodes, "edges": edges}, x


def poly_chain(n_slots, seed=19, n_in=3, degrees=(5, 4)):
    """dense -> polynomial of degree 5 -> dense -> polynomial of degree 4: the
    generic-degree activation (Chebyshev-like random coefficients)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    blocks = []
    for d in degrees:
        Wm = rng.normal(0.0, np.sqrt(1.0 / n_in), size=(n_in, n_in))
        blocks.append(_linear(*dense_csr(Wm), rng.normal(0.0, 0.1, size=n_in)))
        a = list(rng.normal(0.0, 0.3, size=d + 1) / (1.0 + np.arange(d + 1)))
        blocks.append({"kind": "poly", "coeffs": a})
    g = chain_graph(n_in, blocks)
    x = rng.uniform(-1.0, 1.0, size=(n_in, n_slots))
    return g, x


def deep_mlp(n_slots, seed=13, n_in=4, hidden=4, n_out=2):
    """Multiplicative depth 8 (dense, sigmoid fit, dense, sigmoid fit, dense,
    square), so Alg. parameterise asks for N = 32768 and [60, 40 x 8, 60]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W0 = rng.normal(0.0, np.sqrt(2.0 / (n_in + hidden)), size=(hidden, n_in))
    W1 = rng.normal(0.0, np.sqrt(2.0 / (2 * hidden)), size=(hidden, hidden))
    W2 = rng.normal(0.0, np.sqrt(2.0 / (hidden + n_out)), size=(n_out, hidden))
    sig = sigmoid_fit()
    g = chain_graph(n_in, [
        _linear(*dense_csr(W0), rng.normal(0.0, 0.1, size=hidden)),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W1), np.zeros(hidden)),
        {"kind": "poly", "coeffs": sig},
        _linear(*dense_csr(W2), np.zeros(n_out)),
        {"kind": "square"},
    ])
    x = rng.uniform(-1.0, 1.0, size=(n_in, n_slots))
    return g, x


def branch_graph(n_slots, seed=11, n_in=3, n_mid=4):
    """Two inputs on paths of different depth meeting at an 'add' node (the
    x0 / x1 situation of Fig. fhe_parm_problem: x1 meets two computations,
    x0 one): x1 -> linear -> linear -> add, x0 -> linear -> add, then
    add -> square -> output.  The shallower branch is level-matched by
    mod-drop at the add."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Wa = rng.normal(0.0, 0.5, size=(n_mid, n_in))
    Wb = rng.normal(0.0, 0.5, size=(n_mid, n_mid))
    Wc = rng.normal(0.0, 0.5, size=(n_mid, n_in))
    nodes = [
        {"kind": "input", "n": n_in},                                   # 0: x0
        {"kind": "input", "n": n_in},                                   # 1: x1
        _linear(*dense_csr(Wa), rng.normal(0, 0.1, n_mid)),             # 2: c0
        _linear(*dense_csr(Wb), rng.normal(0, 0.1, n_mid)),             # 3: c1 (x1)
        _linear(*dense_csr(Wc), rng.normal(0, 0.1, n_mid)),             # 4: c1 (x0)
        {"kind": "add"},                                                # 5
        {"kind": "square"},                                             # 6
        {"kind": "output"},                                             # 7
    ]
    edges = [(1, 2), (2, 3), (0, 4), (3, 5), (4, 5), (5, 6), (6, 7)]
    x0 = rng.uniform(-1, 1, size=(n_in, n_slots))
    x1 = rng.uniform(-1, 1, size=(n_in, n_slots))
    return {"nodes": nodes, "edges": edges}, [x0, x1]


def input_nodes(graph):
    return [i for i, n in enumerate(graph["nodes"]) if n["kind"] == "input"]


def output_nodes(graph):
    return [i for i, n in enumerate(graph["nodes"]) if n["kind"] == "output"]
