"""FP64 oracle of partitioned_contract on arbitrary graphs (TEST INFRASTRUCTURE).

Plain restatement of Algorithm partitioned_contract (Sec. 3.2) for the
maximally unbalanced path that the paper's experiments use on lattices and
random regular graphs (Sec. 7.3): the intermediate I_s = V_0 u .. u V_s
absorbs the next part V_{s+1}; every intermediate with open edges is
approximated by an MPS embedding tree (App. C) with Algorithm
approx_tensor_network (Sec. 6), i.e. ceil(d / r) passes of
density_matrix_alg (Sec. 5); the last absorption closes the network.

Steps of the plan (graph only, never tensor data):
  * edge sets E(V_a, V_b) between two parts (Algorithm partitioned_contract),
    each ordered by (vertex in the earlier part, vertex in the later part,
    edge id);
  * reference ordering tau_s of the open edge sets of I_s;
  * constraint tree of the open edge sets from the parts still to come
    (the construction of the appendix on the constraint tree);
  * sigma_s = Algorithm linear_ordering_under_constraint_tree (Kendall-Tau
    minimisation over the children of every constraint-tree node);
  * d = Kendall-Tau distance(tau_s, sigma_s), ceil(d / r) passes whose
    edge-set orderings are equally spaced (r adjacent swaps apart) on the
    bubble-sort path from tau_s to sigma_s;
  * every pass contracts the tensors embedded at each tree vertex first
    ("contract T(v) first", Sec. 5.3): the network is laid along the MPS
    tree's chain of leaves, each tensor at one chain position, and an edge
    between positions p < q passes through the blocks in between (a delta).

Readings where the paper is silent (listed in the design notes):
  * tau_s: tau_1 orders the edge sets of I_1 by their later part with the
    sets of V_1 first; tau_s (s >= 2) is sigma_{s-1} with the sets into V_s
    removed and V_s's own sets (by later part) inserted where the first
    removed set stood (the MPS keeps its order, the part takes the place of
    the legs it absorbs).
  * constraint tree: node i (the i-th part still to come) joins the sets
    between I_s and that part and the subtrees of the earlier nodes j whose
    parts are adjacent to it; a node with one child is that child; every
    node is unordered; the roots left at the end join under one root.
  * Kendall-Tau minimisation over the permutations of a node's children:
    exact (subset dynamic programme, ties to the lexicographically smallest
    permutation of the children sorted by their first tau position) for at
    most 12 children, else the children sorted by mean tau position.
  * embedding phi: a tensor owning an open leg sits at the reference
    position of its first leg; MPS sites whose leg is absorbed spread
    evenly over the positions of the new legs; tensors without legs take
    the smallest position among their placed neighbours (repeated rounds).
    phi changes the cost, never the result (each L_v is defined by the
    whole network).
  * an intermediate with fewer than 3 open edges absorbs the next part too.
  * ranks r_0 = d_0, r_k = min(chi, r_{k-1} d_k, D_k, prod_{j>k} d_j).
"""
import numpy as np

from . import dmtree


# ------------------------------------------------------------------ the graph

class _Graph:
    def __init__(self, n, edges, dims):
        self.n = int(n)
        self.edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
        self.dims = [int(x) for x in dims]
        self.inc = [[] for _ in range(self.n)]
        for e, (u, v) in enumerate(self.edges):
            self.inc[int(u)].append(e)
            self.inc[int(v)].append(e)
        for lst in self.inc:
            lst.sort()

    def other(self, e, v):
        u, w = int(self.edges[e][0]), int(self.edges[e][1])
        return w if u == v else u


def parts_from_env(n, env_size):
    """Consecutive runs of env_size vertex ids (the last run may be shorter)."""
    return [list(range(i, min(n, i + env_size))) for i in range(0, n, env_size)]


def _merge_small(g, parts):
    """Merge V_{s+1} into V_s while I_s would have fewer than 3 open edges."""
    parts = [sorted(p) for p in parts]
    s = 1
    while s <= len(parts) - 2:
        inside = set(v for p in parts[: s + 1] for v in p)
        n_open = sum(1 for (u, v) in g.edges if (int(u) in inside) != (int(v) in inside))
        if n_open < 3:
            parts[s] = sorted(parts[s] + parts[s + 1])
            del parts[s + 1]
        else:
            s += 1
    return parts


# ------------------------------------------------------ Kendall-Tau machinery

def kt_distance(a, b):
    """Kendall-Tau distance (Def. Kendall-Tau distance): pairs ordered
    differently in the two orderings of the same elements."""
    pos = {x: i for i, x in enumerate(b)}
    seq = [pos[x] for x in a]
    return sum(1 for i in range(len(seq)) for j in range(i + 1, len(seq)) if seq[i] > seq[j])


def _best_permutation(children, tau_pos):
    """Order of the children (lists of edge sets, each in fixed order) whose
    concatenation is closest to tau in Kendall-Tau distance."""
    m = len(children)
    if m <= 1:
        return list(range(m))
    cross = [[0] * m for _ in range(m)]       # cross[x][y]: x before y costs this
    for x in range(m):
        for y in range(m):
            if x != y:
                cross[x][y] = sum(1 for e in children[x] for f in children[y]
                                  if tau_pos[f] < tau_pos[e])
    if m > 12:
        def key(x):
            return (sum(tau_pos[e] for e in children[x]), len(children[x]))
        order = list(range(m))
        # mean position, exact rational comparison, ties by first position
        import functools

        def cmp(x, y):
            sx, nx = key(x)
            sy, ny = key(y)
            if sx * ny != sy * nx:
                return -1 if sx * ny < sy * nx else 1
            return -1 if x < y else (1 if x > y else 0)
        return sorted(order, key=functools.cmp_to_key(cmp))
    full = (1 << m) - 1
    g = [0] * (1 << m)
    for S in range(full - 1, -1, -1):
        best = None
        for x in range(m):
            if S >> x & 1:
                continue
            rest = full & ~S & ~(1 << x)
            c = sum(cross[x][y] for y in range(m) if rest >> y & 1) + g[S | (1 << x)]
            if best is None or c < best:
                best = c
        g[S] = best
    order, S = [], 0
    while S != full:
        for x in range(m):
            if S >> x & 1:
                continue
            rest = full & ~S & ~(1 << x)
            c = sum(cross[x][y] for y in range(m) if rest >> y & 1) + g[S | (1 << x)]
            if c == g[S]:
                order.append(x)
                S |= 1 << x
                break
    return order


# ------------------------------------------------ orderings of the edge sets

def _constraint_order(tau, s, N, adj_parts):
    """sigma_s: Algorithm linear_ordering_under_constraint_tree on the open
    edge sets ``tau`` of I_s (reference ordering tau), constraint tree from the
    parts s+1 .. N-1 still to come."""
    tau_pos = {k: i for i, k in enumerate(tau)}
    # tree elements: ("leaf", set) or ("node", idx); children lists per node
    parent = {}
    children = {}
    rep = {}
    n_nodes = 0

    def top(x):
        while x in parent:
            x = parent[x]
        return x

    for i in range(1, N - s):
        b = s + i
        kids = [("leaf", k) for k in tau if k[1] == b]
        for j in range(1, i):
            if (s + j) in adj_parts[b] and rep.get(j) is not None:
                kids.append(top(rep[j]))
        seen, uniq = set(), []
        for x in kids:
            if x not in seen:
                seen.add(x)
                uniq.append(x)
        if len(uniq) >= 2:
            node = ("node", n_nodes)
            n_nodes += 1
            children[node] = uniq
            for x in uniq:
                parent[x] = node
            rep[i] = node
        elif len(uniq) == 1:
            rep[i] = uniq[0]
        else:
            rep[i] = None
    roots, seen = [], set()
    for k in tau:
        t = top(("leaf", k))
        if t not in seen:
            seen.add(t)
            roots.append(t)
    if len(roots) == 1:
        root = roots[0]
    else:
        root = ("node", n_nodes)
        children[root] = roots

    def order_of(x):                            # post-order DFS
        if x[0] == "leaf":
            return [x[1]]
        subs = [order_of(c) for c in children[x]]
        subs.sort(key=lambda o: min(tau_pos[k] for k in o))
        perm = _best_permutation(subs, tau_pos)
        out = []
        for p in perm:
            out.extend(subs[p])
        return out

    return order_of(root)


def _swap_path(tau, sigma, r, n_pass):
    """Orderings after min(p r, d) adjacent swaps (p = 1..n_pass) on the
    bubble-sort path from tau to sigma (left-to-right sweeps)."""
    rank = {k: i for i, k in enumerate(sigma)}
    seq = list(tau)
    snaps = [list(seq)]
    changed = True
    while changed:
        changed = False
        for i in range(len(seq) - 1):
            if rank[seq[i]] > rank[seq[i + 1]]:
                seq[i], seq[i + 1] = seq[i + 1], seq[i]
                snaps.append(list(seq))
                changed = True
    d = len(snaps) - 1
    return [snaps[min(p * r, d)] for p in range(1, n_pass + 1)]


# ---------------------------------------------------------- chain layout

def _label_key(lab):
    return (0 if lab[0] == "b" else 1, lab[1])


def capacity(dim):
    """Integer cut weight of an edge: round(2^16 log2 dim) (w(e) = ln s of
    Sec. 2.1 up to a constant factor, in exact integers)."""
    import math
    return int(round(65536.0 * math.log2(dim)))


def _min_cut_source_side(n_nodes, arcs, sources, sinks):
    """Inclusion-minimal source side of a minimum cut (the nodes reachable
    from the sources in the residual graph of a maximum flow).  arcs: list of
    (a, b, cap) undirected edges; sources/sinks: terminal node lists."""
    INF = 1 << 60
    s, t = n_nodes, n_nodes + 1
    cap = {}
    nbr = [set() for _ in range(n_nodes + 2)]

    def add(a, b, c):
        cap[(a, b)] = cap.get((a, b), 0) + c
        cap.setdefault((b, a), 0)
        nbr[a].add(b)
        nbr[b].add(a)

    for a, b, c in arcs:
        add(a, b, c)
        add(b, a, c)
    for x in sources:
        add(s, x, INF)
    for x in sinks:
        add(x, t, INF)
    while True:                      # Edmonds-Karp: shortest augmenting paths
        prev = {s: None}
        queue = [s]
        head = 0
        while head < len(queue) and t not in prev:
            x = queue[head]
            head += 1
            for y in sorted(nbr[x]):
                if y not in prev and cap[(x, y)] > 0:
                    prev[y] = x
                    queue.append(y)
        if t not in prev:
            return set(prev) - {s}
        f, y = INF, t
        while prev[y] is not None:
            f = min(f, cap[(prev[y], y)])
            y = prev[y]
        y = t
        while prev[y] is not None:
            cap[(prev[y], y)] -= f
            cap[(y, prev[y])] += f
            y = prev[y]


def _layout(tensors, legs, dim, leaves, n_pos):
    """Embedding phi of the tensors along the MPS tree's chain (Algorithm
    tree_embedding: at every tree edge, a minimum cut between the leaves on
    its two sides).  With leaves (a DM pass), leaf slot j sits at position j;
    without (the closing chain), the MPS sites ("s", k) are the terminals at
    position k.  Cut k separates positions <= k from > k; the inclusion-
    minimal minimum cuts are nested in k, so phi(t) is the first cut whose
    source side holds t.  Returns phi, the labels crossing every cut (ordered
    by label key) and the cut dims D (D_{n-1} = 1)."""
    where = {}
    for t in tensors:
        for lab in legs[t]:
            where.setdefault(lab, []).append(t)
    idx = {t: i for i, t in enumerate(tensors)}
    nt = len(tensors)
    arcs = []
    for lab, ts in where.items():
        c = capacity(dim[lab])
        if len(ts) == 2:
            arcs.append((idx[ts[0]], idx[ts[1]], c))
    slot = {}
    if leaves:
        for j, lab in enumerate(leaves):
            if len(where.get(lab, [])) != 1:
                raise ValueError("leaf %r must have one owner" % (lab,))
            slot[lab] = nt + j
            arcs.append((idx[where[lab][0]], nt + j, capacity(dim[lab])))
        n_nodes = nt + len(leaves)
        term = [nt + j for j in range(len(leaves))]
    else:
        n_nodes = nt
        term = [idx[("s", k)] for k in range(n_pos)]
    for lab, ts in where.items():
        if len(ts) == 1 and lab not in slot:
            raise ValueError("dangling edge %r" % (lab,))
    phi = {}
    for k in range(n_pos - 1):
        left = _min_cut_source_side(n_nodes, arcs, term[: k + 1], term[k + 1:])
        for t in tensors:
            if t not in phi and idx[t] in left:
                phi[t] = k
    for t in tensors:
        phi.setdefault(t, n_pos - 1)
    pi = {lab: i for i, lab in enumerate(leaves)}
    cross = [[] for _ in range(max(n_pos - 1, 0))]
    for lab, ts in where.items():
        if len(ts) == 2:
            a, b = phi[ts[0]], phi[ts[1]]
        else:
            a, b = phi[ts[0]], pi[lab]
        for k in range(min(a, b), max(a, b)):
            cross[k].append(lab)
    for c in cross:
        c.sort(key=_label_key)
    D = [int(np.prod([dim[lab] for lab in c])) if c else 1 for c in cross] + [1]
    return phi, cross, D


# ---------------------------------------------------------------- the plan

def plan(n, edges, dims, parts, chi, swap_batch=0):
    """Plan of partitioned_contract on the maximally unbalanced path over
    ``parts`` (vertex lists in path order).  chi: int, or a function
    chi(step, pass, k) for per-edge ranks.  swap_batch r <= 0: one pass.

    Returns dict(parts, steps): every step but the last has 'passes', each
    pass dict(leaves, d, D, r, phi, cross, tensors, legs, dim, n_swaps); the
    last step ('close') has phi, cross, D of the closing chain."""
    g = _Graph(n, edges, dims)
    seen = sorted(v for p in parts for v in p)
    if seen != list(range(g.n)):
        raise ValueError("parts must cover every vertex once")
    parts = _merge_small(g, parts)
    N = len(parts)
    if N < 3:
        raise ValueError("need at least one approximated intermediate")
    part_of = [0] * g.n
    for i, p in enumerate(parts):
        for v in p:
            part_of[v] = i
    sets, adj_parts = {}, [set() for _ in range(N)]
    for e, (u, v) in enumerate(g.edges):
        a, b = sorted((part_of[int(u)], part_of[int(v)]))
        if a == b:
            continue
        sets.setdefault((a, b), []).append(e)
        adj_parts[a].add(b)
        adj_parts[b].add(a)

    def in_part(e, p):
        u, v = int(g.edges[e][0]), int(g.edges[e][1])
        return u if part_of[u] == p else v

    for (a, b), lst in sets.items():
        lst.sort(key=lambda e: (in_part(e, a), in_part(e, b), e))

    def expand(order):
        return [("g", e) for k in order for e in sets[k]]

    dim = {("g", e): g.dims[e] for e in range(len(g.edges))}
    sigma = sorted([k for k in sets if k[0] == 0], key=lambda k: k[1])
    mps = None                     # (leaf labels, bond dims) of the current MPS
    steps = []
    for s in range(1, N):
        if s == 1:
            raw = parts[0] + parts[1]
        else:
            raw = list(parts[s])
        raw_t = [("v", v) for v in sorted(raw)]
        legs = {t: [("g", e) for e in g.inc[t[1]]] for t in raw_t}
        site_t = []
        mps_leaf = {}
        if mps is not None:
            leaves_in, bonds = mps
            m = len(leaves_in)
            for k in range(m):
                t = ("s", k)
                site_t.append(t)
                lg = []
                if k >= 1:
                    lg.append(("b", k - 1))
                lg.append(leaves_in[k])
                if k <= m - 2:
                    lg.append(("b", k))
                legs[t] = lg
                mps_leaf[k] = leaves_in[k]
            for k, r in enumerate(bonds):
                dim[("b", k)] = r
        tensors = site_t + raw_t
        if s == N - 1:
            phi, cross, D = _layout(tensors, legs, dim, [], len(site_t))
            steps.append(dict(close=True, phi=phi, cross=cross, D=D, tensors=tensors,
                              legs=legs, dim=dict(dim)))
            break
        removed = [i for i, k in enumerate(sigma) if k[1] == s]
        new = sorted([k for k in sets if k[0] == s], key=lambda k: k[1])
        kept = [k for k in sigma if k[1] != s]
        at = removed[0] if removed else len(kept)
        tau = kept[:at] + new + kept[at:]
        sig = _constraint_order(tau, s, N, adj_parts)
        d_kt = kt_distance(tau, sig)
        if swap_batch and swap_batch > 0:
            n_pass = max(1, -(-d_kt // swap_batch))
            orders = _swap_path(tau, sig, swap_batch, n_pass)
        else:
            orders = [sig]
        passes = []
        ref = expand(tau)
        for p, order in enumerate(orders):
            leaves = expand(order)
            ref_pos = {lab: i for i, lab in enumerate(ref)}
            phi, cross, D = _layout(tensors, legs, dim, leaves, len(leaves))
            nl = len(leaves)
            d = [dim[lab] for lab in leaves]
            r = [d[0]]
            for k in range(1, nl - 1):
                beyond = int(np.prod(d[k + 1:]))
                chi_k = chi(s, p, k) if callable(chi) else chi
                r.append(int(min(chi_k, r[k - 1] * d[k], D[k], beyond)))
            passes.append(dict(leaves=leaves, d=d, D=D, r=r, phi=phi, cross=cross,
                               tensors=tensors, legs=legs, dim=dict(dim), n_kt=d_kt))
            # the next pass sees only the MPS this pass writes
            site_t = [("s", k) for k in range(nl)]
            legs = {}
            mps_leaf = {}
            for k in range(nl):
                lg = []
                if k >= 1:
                    lg.append(("b", k - 1))
                lg.append(leaves[k])
                if k <= nl - 2:
                    lg.append(("b", k))
                legs[("s", k)] = lg
                mps_leaf[k] = leaves[k]
            for k in range(nl - 1):
                dim[("b", k)] = r[k]
            tensors = site_t
            ref = leaves
        mps = (passes[-1]["leaves"], passes[-1]["r"])
        steps.append(dict(close=False, passes=passes, tau=tau, sigma=sig))
        sigma = sig
    return dict(parts=parts, steps=steps)


# ------------------------------------------------------------ the contraction

def _contract_pairwise(ops, out):
    """Contraction of the operands ops = [array, labels, array, labels, ...]
    into the labels ``out`` by repeated pairwise tensordot: the pair sharing
    a label whose result is smallest first (an outer product only when no pair
    shares one)."""
    items = [(np.asarray(ops[i]), list(ops[i + 1])) for i in range(0, len(ops), 2)]
    if not items:
        return np.ones(())
    while len(items) > 1:
        best = None
        for i in range(len(items)):
            for j in range(i + 1, len(items)):
                (a, la), (b, lb) = items[i], items[j]
                shared = [l for l in la if l in lb]
                keep = [l for l in la if l not in shared] + [l for l in lb if l not in shared]
                size = 1
                for l in keep:
                    size *= (a.shape[la.index(l)] if l in la else b.shape[lb.index(l)])
                key = (0 if shared else 1, size, i, j)
                if best is None or key < best[0]:
                    best = (key, i, j, shared, keep)
        _, i, j, shared, keep = best
        (a, la), (b, lb) = items[i], items[j]
        c = np.tensordot(a, b, axes=([la.index(l) for l in shared], [lb.index(l) for l in shared]))
        items = [it for q, it in enumerate(items) if q not in (i, j)] + [(c, keep)]
    y, ly = items[0]
    extra = [l for l in ly if l not in out]
    if extra:
        raise ValueError("labels left uncontracted")
    return np.transpose(y, [ly.index(l) for l in out]) if out else y


def _block(k, pas, arrays, leaves, n_pos):
    """Y_k of the chain: the tensors at position k contracted together, an
    identity (delta) for every edge passing through, shaped (D_{k-1}, d_k, D_k)
    (d_k = 1 on the closing chain)."""
    cross, phi, legs, dim = pas["cross"], pas["phi"], pas["legs"], pas["dim"]
    left = cross[k - 1] if k >= 1 else []
    right = cross[k] if k < n_pos - 1 else []
    lset, rset = set(left), set(right)
    leaf = leaves[k] if leaves else None
    ids = {}

    def lid(key):
        if key not in ids:
            ids[key] = len(ids)
        return ids[key]

    ops, core = [], []
    for t in pas["tensors"]:
        if phi[t] != k:
            continue
        sub = []
        for lab in legs[t]:
            if lab in lset:
                key = ("L", lab)
            elif lab in rset:
                key = ("R", lab)
            elif lab == leaf:
                key = ("X",)
            else:
                key = ("I", lab)
            sub.append(lid(key))
            if key[0] != "I":
                core.append(key)
        ops += [arrays[t], sub]
    # the tensors at k, summed over their internal edges
    y = _contract_pairwise(ops, [ids[key] for key in core])
    labels = list(core)
    # a delta for every edge passing through, and for a leaf whose owner sits
    # at another position
    for lab in left:
        if lab in rset:
            y = np.multiply.outer(y, np.eye(dim[lab]))
            labels += [("L", lab), ("R", lab)]
    if leaf is not None and ("X",) not in labels:
        side = "L" if leaf in lset else "R"
        y = np.multiply.outer(y, np.eye(dim[leaf]))
        labels += [(side, leaf), ("X",)]
    out = [("L", lab) for lab in left]
    if leaf is not None:
        out.append(("X",))
    out += [("R", lab) for lab in right]
    y = np.transpose(y, [labels.index(key) for key in out]) if out else y
    Dl = int(np.prod([dim[lab] for lab in left])) if left else 1
    Dr = int(np.prod([dim[lab] for lab in right])) if right else 1
    dk = dim[leaf] if leaf is not None else 1
    return np.asarray(y, dtype=np.float64).reshape(Dl, dk, Dr)


def _site_arrays(U, Mr, leaves, r):
    """MPS sites of a pass's output as arrays whose axes follow the site's
    legs ([left bond], leaf, [right bond])."""
    n = len(leaves)
    d = [None] * n
    S = {}
    d0 = r[0]
    S[("s", 0)] = np.eye(d0)                                    # (leaf, b_0)
    for k in range(1, n - 1):
        rp = r[k - 1]
        S[("s", k)] = U[k].reshape(rp, -1, r[k])               # (b_{k-1}, leaf, b_k)
    S[("s", n - 1)] = Mr.reshape(r[n - 2], -1)                 # (b_{n-2}, leaf)
    return S


def partitioned_contract_graph(workload, parts, chi, swap_batch=0, trace=None):
    """ln Z of a closed Ising (or any) network by the plan above.

    workload: dict(n, edges, tensors) with site tensors whose legs follow the
    ascending incident-edge ids; parts: vertex lists in path order.
    Returns dict(logz, sign, logscale, plan)."""
    n = workload["n"]
    edges = np.asarray(workload["edges"], dtype=np.int64)
    dims = []
    inc = [[] for _ in range(n)]
    for e, (u, v) in enumerate(edges):
        inc[int(u)].append(e)
        inc[int(v)].append(e)
    for e in range(len(edges)):
        u = int(edges[e][0])
        pos = sorted(inc[u]).index(e)
        dims.append(np.asarray(workload["tensors"][u]).shape[pos])
    P = plan(n, edges, dims, parts, chi, swap_batch)
    logscale = 0.0
    raw = {}
    for v in range(n):
        t = np.asarray(workload["tensors"][v], dtype=np.float64)
        nrm = np.linalg.norm(t)
        logscale += np.log(nrm)
        raw[("v", v)] = t / nrm
    mps = {}
    for st in P["steps"]:
        if st["close"]:
            arrays = dict(raw)
            arrays.update(mps)
            m = len(st["D"])
            vec = np.ones((1,))
            for k in range(m):
                y = _block(k, st, arrays, None, m)[:, 0, :]
                vec = vec @ y
                mx = np.max(np.abs(vec))
                if mx > 0:
                    logscale += np.log(mx)
                    vec = vec / mx
            s = float(vec.reshape(-1)[0])
            if not s > 0:
                return dict(logz=float("nan"), sign=float(np.sign(s)), logscale=logscale, plan=P)
            return dict(logz=float(np.log(s) + logscale), sign=1.0, logscale=logscale, plan=P)
        for p_i, pas in enumerate(st["passes"]):
            arrays = dict(raw)
            arrays.update(mps)
            leaves = pas["leaves"]
            nl = len(leaves)
            Y = [_block(k, pas, arrays, leaves, nl) for k in range(nl)]
            blocks = [None] * nl
            blocks[1] = np.einsum("aib,bjc->ijc", Y[0], Y[1])
            for k in range(2, nl):
                blocks[k] = Y[k]
            r = pas["r"]
            rec = [] if trace is not None else None
            U, Mr, lognorm = dmtree.density_matrix_alg(blocks, lambda v, r=r: r[v], trace=rec)
            logscale += lognorm
            for k in range(1, nl - 1):
                if U[k].shape[1] != r[k]:
                    raise AssertionError("rank differs from the plan")
            mps = _site_arrays(U, Mr, leaves, r)
            if trace is not None:
                trace.append(dict(pas=pas, U=U, Mr=Mr, lognorm=lognorm, vertices=rec, Y=Y))
    raise AssertionError("plan without a closing step")
