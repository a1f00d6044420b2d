"""protosim -- a step-by-step model of the paper's signalling machinery, on the CPU.

TEST INFRASTRUCTURE ONLY (imported by tests; never by the library).  Pure Python,
for small streams.  It is written independently of oracle/rs_oracle.c: its stage
arithmetic is re-derived here, so agreement between the two pins both.

What it models (Timcheck & Buhler):
  * Section 2.1 -- a linear pipeline of nodes joined by fixed-capacity data queues;
    a non-preemptive scheduler repeatedly fires some node with pending input until
    none is left.  Here the choice among fireable nodes is random (seeded), so the
    tests exercise many schedules.
  * Section 2.2 -- one pipeline instance per processor; processors compete for a
    common input through an atomic cursor (here: units of K consecutive parents).
    A firing consumes an ensemble of at most W items.
  * Section 3.1 -- a signal queue beside each data queue and the credit protocol:
      sender rule 1: signal queue empty -> credit = items now in the data queue;
      sender rule 2: otherwise -> credit = items emitted since the previous signal
                     (a counter reset whenever a signal is emitted);
      receiver rule 1: no signal queued -> consume data freely;
      receiver rule 2a: counter > 0 -> consume at most `counter` items, decrementing;
      receiver rule 2b: counter == 0 -> move the head signal's credit to the counter
                        if it has any, else consume the head signal.
  * Section 3.2 -- two-phase firing (data phase limited by queued items, downstream
    space and, with a signal pending, the counter; then a signal phase while the
    counter is 0) and fireability from a-priori maximum fan-out.
  * Section 3.3 -- the SIMD rule: an ensemble never exceeds the counter when a
    signal is pending, so no ensemble straddles a signal.
  * Section 4 -- enumeration emits Begin(r), the elements of parent r, End(r);
    downstream nodes switch their parent context on Begin; the aggregate resets on
    Begin and emits one result on End (Figure 4's begin/run/end).
  * The in-band alternative of Section 2.3 / Section 5 ("tag"): every item carries
    its region id, there are no signals and ensembles may mix regions.

Checks it records for the tests: each edge's receive order equals its send order
with signals in place (Lemma 1), the run ends with every queue empty (Lemma 2),
counter > 0 implies pending data at every step (first claim of Lemma 2's proof),
every ensemble holds items of one region only and sees that region's context
(signal strategy), each region gets exactly one aggregate.
"""
from __future__ import annotations

import random
from collections import deque

M32 = 0xFFFFFFFF
IDENT = (0, 0, M32)          # (count, sum, min) of an empty region


# ---- stage arithmetic, restated from the operation definitions --------------

def fmix32(h):
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M32
    h ^= h >> 16
    return h


def hash32(a, b):
    return fmix32((a ^ fmix32((b ^ 0x9E3779B9) & M32)) & M32)


def apply_op(st, x, parent, t):
    """Outputs (a list of 0..k values) of element-stage `st` for input x."""
    name = st[0]
    if name == "filter_mod":
        return [x] if x % st[1] == st[2] else []
    if name == "filter_hash_ctx":
        return [x] if (hash32(x, st[1]) ^ t) < st[2] else []
    if name == "filter_weight_lt":
        return [x] if hash32(x, st[1]) < hash32(parent, st[1]) else []
    if name == "map_mul":
        return [(st[1] * x + st[2]) & M32]
    if name == "expand":
        k, salt = st[1], st[2]
        n = hash32(x, salt) % (k + 1)
        return [hash32(x, (salt + 1 + j) & M32) for j in range(n)]
    raise ValueError(name)


def max_fanout(st):
    return st[1] if st[0] == "expand" else 1


# ---- queues -----------------------------------------------------------------

class Edge:
    def __init__(self, cap_q, cap_s):
        self.q = deque()            # data items: (value, true_region, tag)
        self.s = deque()            # signals: [kind, region, credit]
        self.cap_q, self.cap_s = cap_q, cap_s
        self.emitted = 0            # sender's counter, reset on each signal
        self.sent = []              # send log: ('d', value) / ('s', kind, region)
        self.recv = []              # receive log, same format

    def push_item(self, item):
        assert len(self.q) < self.cap_q, "data queue overflow"
        self.q.append(item)
        self.emitted += 1
        self.sent.append(("d", item[0]))

    def push_signal(self, kind, region):
        assert len(self.s) < self.cap_s, "signal queue overflow"
        credit = len(self.q) if not self.s else self.emitted     # sender rules 1 / 2
        self.s.append([kind, region, credit])
        self.emitted = 0
        self.sent.append(("s", kind, region))


class Node:
    def __init__(self, st, ein, eout):
        self.st, self.ein, self.eout = st, ein, eout
        self.credit = 0
        self.parent = None          # region id of the current context (signal strategy)
        self.ensembles = []         # sizes of ensembles fired


class Processor:
    def __init__(self, pipeline, W, cap_q, cap_s, strategy):
        n = len(pipeline)
        self.pipeline = pipeline
        self.W, self.strategy = W, strategy
        self.edges = [Edge(cap_q, cap_s) for _ in range(n - 1)]
        self.nodes = [None] + [Node(pipeline[i], self.edges[i - 1], self.edges[i] if i < n - 1 else None)
                               for i in range(1, n)]
        self.parents = deque()      # claimed parents not yet fully enumerated
        self.enum_pos = 0           # next element index of parents[0]
        self.enum_begun = False
        self.acc = {}               # aggregate accumulators by region (tag strategy)
        self.cur_acc = None         # aggregate accumulator (signal strategy)
        self.cur_region = None


class Sim:
    """Run `pipeline` over `stream` on `n_proc` simulated processors.

    W: ensemble width; cap_q/cap_s: data/signal queue capacities; K: parents claimed
    per cursor step; strategy: "signal" or "tag"; seed: scheduler randomness."""

    def __init__(self, pipeline, stream, *, W=4, cap_q=8, cap_s=4, K=2, n_proc=1,
                 strategy="signal", seed=0, max_steps=10_000_000):
        worst = max([max_fanout(s) for s in pipeline[1:-1]] + [1])
        if cap_q < W * worst:
            raise ValueError("data queue smaller than one ensemble's worst-case output")
        if cap_s < 2:
            raise ValueError("signal queue must hold a Begin/End pair")
        self.pipeline, self.stream = pipeline, stream
        self.W, self.K, self.strategy = W, K, strategy
        self.rng = random.Random(seed)
        self.procs = [Processor(pipeline, W, cap_q, cap_s, strategy) for _ in range(n_proc)]
        self.cursor = 0
        self.R = int(stream["R"])
        self.results = {}
        self.result_writes = [0] * self.R
        self.violations = []
        self.steps = 0
        self.max_steps = max_steps
        L = stream.get("len")
        off = stream.get("offsets")
        if off is not None:
            self.off = [int(v) for v in off]
        else:
            self.off = [0]
            for v in L:
                self.off.append(self.off[-1] + int(v))

    # -- stream access
    def parent_id(self, r):
        p = self.stream.get("parents")
        return int(p[r]) if p is not None else r

    def ctx(self, r):
        c = self.stream.get("ctx")
        return int(c[r]) if c is not None else 0

    def element(self, r, i):
        if self.pipeline[0][0] == "enum_hash":
            return hash32(self.parent_id(r), i)
        return int(self.stream["elements"][self.off[r] + i])

    def length(self, r):
        return self.off[r + 1] - self.off[r]

    # -- fireability (Section 3.2)
    def enum_fireable(self, P):
        e = P.edges[0]
        has_input = bool(P.parents) or self.cursor < self.R
        return has_input and len(e.q) < e.cap_q and len(e.s) < e.cap_s - 1

    def node_fireable(self, P, i):
        nd = P.nodes[i]
        if not nd.ein.q and not nd.ein.s:
            return False
        if nd.eout is None:
            return True
        k = max_fanout(nd.st)
        return nd.eout.cap_q - len(nd.eout.q) >= k and len(nd.eout.s) < nd.eout.cap_s

    # -- enumeration
    def fire_enum(self, P):
        e = P.edges[0]
        if not P.parents:
            b = self.cursor
            self.cursor = min(self.R, b + self.K)             # atomic claim of K parents
            P.parents.extend(range(b, self.cursor))
            P.enum_pos, P.enum_begun = 0, False
        while P.parents:
            r = P.parents[0]
            if self.strategy == "signal" and not P.enum_begun:
                if len(e.s) >= e.cap_s:
                    return
                e.push_signal("B", r)
            P.enum_begun = True
            L = self.length(r)
            while P.enum_pos < L and len(e.q) < e.cap_q:
                x = self.element(r, P.enum_pos)
                e.push_item((x, r, r if self.strategy == "tag" else None))
                P.enum_pos += 1
            if P.enum_pos < L:
                return                                       # resumes on a later firing
            if self.strategy == "signal":
                if len(e.s) >= e.cap_s:
                    return
                e.push_signal("E", r)
            else:
                # tag strategy: every claimed region still owes one aggregate
                P.acc.setdefault(r, None)
            P.parents.popleft()
            P.enum_pos, P.enum_begun = 0, False
            if self.rng.random() < 0.5:                      # vary firing granularity
                return

    # -- element nodes and the aggregate
    def consume_items(self, P, nd, items):
        last = nd.eout is None
        for (x, r_true, tag) in items:
            r = tag if self.strategy == "tag" else nd.parent
            if self.strategy == "signal" and r != r_true:
                self.violations.append(("context", nd.st, r, r_true))
            if last:
                if self.strategy == "tag":
                    a = P.acc.get(r) or IDENT
                    P.acc[r] = (a[0] + 1, a[1] + x, min(a[2], x))
                else:
                    a = P.cur_acc
                    P.cur_acc = (a[0] + 1, a[1] + x, min(a[2], x))
            else:
                for y in apply_op(nd.st, x, self.parent_id(r), self.ctx(r)):
                    nd.eout.push_item((y, r_true, tag))

    def emit_result(self, r, acc):
        self.results[r] = acc
        self.result_writes[r] += 1

    def fire_node(self, P, i):
        nd = P.nodes[i]
        ein, eout = nd.ein, nd.eout
        k = max_fanout(nd.st) if eout is not None else 1
        # data phase
        while True:
            avail = len(ein.q)
            limit = nd.credit if ein.s else avail
            space = (eout.cap_q - len(eout.q)) // k if eout is not None else avail
            take = min(avail, limit, space, self.W)
            if take <= 0:
                break
            ens = [ein.q.popleft() for _ in range(take)]
            for it in ens:
                ein.recv.append(("d", it[0]))
            if ein.s:
                nd.credit -= take
            if self.strategy == "signal" and len({it[1] for it in ens}) != 1:
                self.violations.append(("mixed-ensemble", nd.st, [it[1] for it in ens]))
            nd.ensembles.append(take)
            self.consume_items(P, nd, ens)
            if self.rng.random() < 0.3:                      # a firing may stop early
                break
        # signal phase
        while nd.credit == 0 and ein.s:
            sig = ein.s[0]
            if sig[2] > 0:
                nd.credit += sig[2]                          # receiver rule 2b, first half
                sig[2] = 0
                break
            if eout is not None and len(eout.s) >= eout.cap_s:
                break
            ein.s.popleft()                                  # receiver rule 2b, second half
            kind, r = sig[0], sig[1]
            ein.recv.append(("s", kind, r))
            if kind == "B":
                nd.parent = r
                if eout is None:
                    P.cur_acc, P.cur_region = IDENT, r       # begin()
            else:
                if eout is None:
                    if P.cur_region != r:
                        self.violations.append(("end-without-begin", r))
                    self.emit_result(r, P.cur_acc)           # end()
                    P.cur_acc, P.cur_region = None, None
            if eout is not None:
                eout.push_signal(kind, r)                    # forward with fresh credit

    def check_claim1(self):
        for P in self.procs:
            for nd in P.nodes[1:]:
                if nd.credit > 0 and not nd.ein.q:
                    self.violations.append(("credit-without-data", nd.st))

    def flush_tag_results(self, P):
        for r, a in list(P.acc.items()):
            self.emit_result(r, a if a is not None else IDENT)
        P.acc.clear()

    def run(self):
        n = len(self.pipeline)
        while True:
            choices = []
            for pi, P in enumerate(self.procs):
                if self.enum_fireable(P):
                    choices.append((pi, 0))
                for i in range(1, n):
                    if self.node_fireable(P, i):
                        choices.append((pi, i))
            if not choices:
                break
            pi, i = self.rng.choice(choices)
            P = self.procs[pi]
            if i == 0:
                self.fire_enum(P)
            else:
                self.fire_node(P, i)
            self.check_claim1()
            self.steps += 1
            if self.steps > self.max_steps:
                raise RuntimeError("no termination within the step budget")
            if self.strategy == "tag" and not any(P.edges[j].q for j in range(n - 1)) and not P.parents:
                self.flush_tag_results(P)
        for P in self.procs:
            if self.strategy == "tag":
                self.flush_tag_results(P)
            for e in P.edges:
                if e.q or e.s:
                    self.violations.append(("non-empty-queue-at-end",))
        return self

    # -- outputs for the tests
    def aggregates(self):
        import numpy as np
        count = np.zeros(self.R, dtype=np.uint32)
        sm = np.zeros(self.R, dtype=np.uint64)
        mn = np.full(self.R, M32, dtype=np.uint32)
        for r, (c, s, m) in self.results.items():
            count[r], sm[r], mn[r] = c, s, m
        return {"count": count, "sum": sm, "min": mn}

    def edge_logs_match(self):
        return all(e.sent == e.recv for P in self.procs for e in P.edges)

    def ensemble_sizes(self, node_index):
        return [s for P in self.procs for s in P.nodes[node_index].ensembles]


def receiver_trace(data, signals, W=8):
    """Apply the receiver rules alone to a prepared queue state.

    data: list of item labels queued on Q; signals: list of (label, credit) queued on
    S; the current credit counter starts at 0.  Returns the order in which the
    receiving node consumes items and signals, firing with ensembles of <= W until
    both queues are empty."""
    q = deque(data)
    s = deque([list(x) for x in signals])
    counter = 0
    out = []
    guard = 0
    while q or s:
        guard += 1
        if guard > 10_000:
            raise RuntimeError("receiver made no progress")
        limit = counter if s else len(q)
        take = min(len(q), limit, W)
        if take:
            out.append([q.popleft() for _ in range(take)])
            if s:
                counter -= take
        while counter == 0 and s:
            if s[0][1] > 0:
                counter, s[0][1] = s[0][1], 0
                break
            out.append(s.popleft()[0])
    return out
